// geometry.cu -- encoding of the fixed-rate geometry streams and the chunk table (Sec. IV-A);
// the stream layout, quantisers and decoder are in geometry.cuh.
#include "geometry.cuh"

namespace {

// One CTA per chunk: the box of its centres and its largest decoded scale (min / max are exact
// and order-free, so any reduction order gives the same bits); a chunk of padding only is zero.
__global__ void k_chunk_bounds(const float* __restrict__ pos, const float* __restrict__ scale,
                               const int32_t* __restrict__ perm, int64_t ns, int64_t chunk_slots,
                               gsc_chunk* __restrict__ chunk) {
  __shared__ float s_lo[3][256], s_hi[3][256], s_sc[256];
  __shared__ int s_any[256];
  const int64_t c = blockIdx.x;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, sc = -INFINITY;
  int any = 0;
  for (int64_t s = c * chunk_slots + threadIdx.x; s < (c + 1) * chunk_slots && s < ns; s += blockDim.x) {
    const int32_t o = perm[s];
    if (o < 0) continue;
    any = 1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float p = pos[3 * (int64_t)o + a];
      lo[a] = fminf(lo[a], p);
      hi[a] = fmaxf(hi[a], p);
      sc = fmaxf(sc, bf16_val(bf16_rne(scale[3 * (int64_t)o + a])));
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) { s_lo[a][threadIdx.x] = lo[a]; s_hi[a][threadIdx.x] = hi[a]; }
  s_sc[threadIdx.x] = sc;
  s_any[threadIdx.x] = any;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int a = 0; a < 3; a++) {
        s_lo[a][threadIdx.x] = fminf(s_lo[a][threadIdx.x], s_lo[a][threadIdx.x + w]);
        s_hi[a][threadIdx.x] = fmaxf(s_hi[a][threadIdx.x], s_hi[a][threadIdx.x + w]);
      }
      s_sc[threadIdx.x] = fmaxf(s_sc[threadIdx.x], s_sc[threadIdx.x + w]);
      s_any[threadIdx.x] |= s_any[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    gsc_chunk e;
    const bool live = s_any[0] != 0;
    for (int a = 0; a < 3; a++) { e.lo[a] = live ? s_lo[a][0] : 0.0f; e.hi[a] = live ? s_hi[a][0] : 0.0f; }
    e.max_scale = live ? s_sc[0] : 0.0f;
    e.pad = 0.0f;
    chunk[c] = e;
  }
}

__global__ void k_geometry_encode(const float* __restrict__ pos, const float* __restrict__ scale,
                                  const float4* __restrict__ rot, const float* __restrict__ logit,
                                  const int32_t* __restrict__ perm, int64_t ns, int64_t chunk_slots, GeomStreams G) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = perm[s];
    if (o < 0) {
#pragma unroll
      for (int a = 0; a < 3; a++) { G.qpos[3 * s + a] = 0; G.qscale[3 * s + a] = 0; }
      G.qrot[s] = 0;
      G.qlogit[s] = 0;
      continue;
    }
    const gsc_chunk e = G.chunk[s / chunk_slots];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const float ext = gs(e.hi[a], e.lo[a]);
      const float t = ext > 0.0f ? gd(gs(pos[3 * (int64_t)o + a], e.lo[a]), ext) : 0.0f;
      G.qpos[3 * s + a] = (uint16_t)quant_unit(t, 65535.0f);
      G.qscale[3 * s + a] = bf16_rne(scale[3 * (int64_t)o + a]);
    }
    // smallest three: normalise, largest |component| (first on ties) made non-negative
    const float4 q4 = rot[o];
    const float q[4] = {q4.x, q4.y, q4.z, q4.w};
    const float nq = __fsqrt_rn(ga(ga(ga(gm(q[0], q[0]), gm(q[1], q[1])), gm(q[2], q[2])), gm(q[3], q[3])));
    float u[4];
#pragma unroll
    for (int a = 0; a < 4; a++) u[a] = nq > 0.0f ? gd(q[a], nq) : (a == 0 ? 1.0f : 0.0f);
    int m = 0;
#pragma unroll
    for (int a = 1; a < 4; a++) if (fabsf(u[a]) > fabsf(u[m == 0 ? 0 : (m == 1 ? 1 : (m == 2 ? 2 : 3))])) m = a;
    const float um = m == 0 ? u[0] : (m == 1 ? u[1] : (m == 2 ? u[2] : u[3]));
    const float sg = um < 0.0f ? -1.0f : 1.0f;
    uint32_t code = (uint32_t)m;
    int sh = 2;
#pragma unroll
    for (int a = 0; a < 4; a++) {
      if (a == m) continue;
      const float c = sg * u[a];
      code |= quant_unit(ga(gm(c, 0.70710678f), 0.5f), 1022.0f) << sh;
      sh += 10;
    }
    G.qrot[s] = code;
    G.qlogit[s] = (uint8_t)quant_unit(gd(ga(logit[o], 8.0f), 16.0f), 255.0f);
  }
}

}  // namespace

extern "C" size_t gsc_geometry_bytes(int64_t n_slots, int64_t chunk_slots) {
  if (n_slots < 0 || chunk_slots < 16 || chunk_slots % 16) return 0;
  return geom_bytes(n_slots, chunk_slots, nullptr);
}

extern "C" size_t gsc_geometry_layout(int64_t n_slots, int64_t chunk_slots, size_t* offsets) {
  if (n_slots < 0 || chunk_slots < 16 || chunk_slots % 16 || !offsets) return 0;
  return geom_bytes(n_slots, chunk_slots, offsets);
}

extern "C" gsc_status gsc_geometry_encode(gsc_ctx* c, const float* d_pos, const float* d_scale, const float* d_rot,
                                          const float* d_logit, const int32_t* d_perm, int64_t n_slots,
                                          int64_t chunk_slots, uint8_t* d_geom, void* stream) {
  GscRange gsc_range_("gsc_geometry_encode");
  if (!c || n_slots < 0 || n_slots % 16 || chunk_slots < 16 || chunk_slots % 16) return GSC_ERR_INVALID_ARG;
  if (n_slots > 0 && (!d_pos || !d_scale || !d_rot || !d_logit || !d_perm || !d_geom)) return GSC_ERR_INVALID_ARG;
  if (((uintptr_t)d_rot % 16) || ((uintptr_t)d_geom % 256)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  if (n_slots == 0) return GSC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const GeomStreams G = geom_streams(d_geom, n_slots, chunk_slots);
  const int64_t nc = (n_slots + chunk_slots - 1) / chunk_slots;
  gsc_count_launch();
  k_chunk_bounds<<<(unsigned)nc, 256, 0, st>>>(d_pos, d_scale, d_perm, n_slots, chunk_slots, G.chunk);
  GSC_CUDA(cudaGetLastError());
  int64_t grid = ceil_div64(n_slots, 256);
  if (grid > gsc_sm_count() * 16) grid = gsc_sm_count() * 16;
  gsc_count_launch();
  k_geometry_encode<<<(int)grid, 256, 0, st>>>(d_pos, d_scale, reinterpret_cast<const float4*>(d_rot), d_logit, d_perm,
                                               n_slots, chunk_slots, G);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}
