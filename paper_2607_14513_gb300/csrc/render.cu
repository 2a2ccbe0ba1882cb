// render.cu -- splatting renderer over a coded scene (Sec. II: Eq. sigmoid, Eq. covar, Eq. opac,
// Eq. preblend with the premultiplied coefficients of Eq. premult; Fig. GSRend: the colour of
// every Gaussian is decoded from its blocks and evaluated for the camera before blending).
//
// Pipeline on the caller's stream: fused block decode + SH evaluation for the camera centre
// (the premultiplied colour c~ = H~ w(f - p), one view); per Gaussian the EWA splat setup (camera
// depth, 2-D covariance with a 0.3 px^2 low-pass, its inverse, the 3-sigma square's 16 x 16 tile
// rectangle, mu = sigmoid(t)); a stable radix sort of the visible Gaussians by depth; a scan of
// their tile counts in that order; one tile key per overlapped tile, emitted in depth order; a
// stable radix sort by tile (each tile's list stays nearest first); tile ranges; and one CTA per
// tile blending its list front to back, two pixels per thread. The setup's decisions (culling, rectangle, depth order) are taken in
// float with a fixed order of correctly rounded operations, so every implementation of the same
// steps takes them the same way.
#include <math.h>
#include <string.h>

#include "geometry.cuh"
#include "gsc_internal.cuh"

namespace {

#define RTILE 16

struct CamDev {
  float R[9], t[3];
  float fx, fy, cx, cy, near_z;
  int32_t width, height, tiles_x, tiles_y;
};

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float dot3(float a0, float b0, float a1, float b1, float a2, float b2) {
  return fa(fa(fm(a0, b0), fm(a1, b1)), fm(a2, b2));
}

// Splat of Gaussian i (Eq. covar, the EWA projection, its tile rectangle): rec0 = (u, v, mu,
// depth), rec1 = conic scaled for exp2, rec2 = premultiplied colour; rect = tile rectangle [x0, x1)
// x [y0, y1). Returns its tile count (0: culled).
__device__ __forceinline__ uint32_t splat_one(int64_t i, float px, float py, float pz, const float (&s3)[3], float4 q,
                                              float lg, const float* __restrict__ rgb, const CamDev& cam,
                                              float4* __restrict__ rec, int4* __restrict__ rect) {
  uint32_t cnt = 0;
  const float* R = cam.R;
  const float x = fa(dot3(R[0], px, R[1], py, R[2], pz), cam.t[0]);
  const float y = fa(dot3(R[3], px, R[4], py, R[5], pz), cam.t[1]);
  const float z = fa(dot3(R[6], px, R[7], py, R[8], pz), cam.t[2]);
  const float nq = __fsqrt_rn(fa(fa(fa(fm(q.x, q.x), fm(q.y, q.y)), fm(q.z, q.z)), fm(q.w, q.w)));
  if (z > cam.near_z && nq > 0.0f) {
    // Eq. covar: Sigma = R(q) D(s) D(s)^T R(q)^T, q = (w, x, y, z)
    const float qw = fd(q.x, nq), qx = fd(q.y, nq), qy = fd(q.z, nq), qz = fd(q.w, nq);
    float r[9];
    r[0] = fs(1.0f, fm(2.0f, fa(fm(qy, qy), fm(qz, qz))));
    r[1] = fm(2.0f, fs(fm(qx, qy), fm(qw, qz)));
    r[2] = fm(2.0f, fa(fm(qx, qz), fm(qw, qy)));
    r[3] = fm(2.0f, fa(fm(qx, qy), fm(qw, qz)));
    r[4] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qz, qz))));
    r[5] = fm(2.0f, fs(fm(qy, qz), fm(qw, qx)));
    r[6] = fm(2.0f, fs(fm(qx, qz), fm(qw, qy)));
    r[7] = fm(2.0f, fa(fm(qy, qz), fm(qw, qx)));
    r[8] = fs(1.0f, fm(2.0f, fa(fm(qx, qx), fm(qy, qy))));
    float m[9], S[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) m[3 * a + b] = fm(r[3 * a + b], s3[b]);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) S[3 * a + b] = dot3(m[3 * a], m[3 * b], m[3 * a + 1], m[3 * b + 1], m[3 * a + 2], m[3 * b + 2]);
    // Jacobian of the pinhole projection at the centre, times the view rotation
    const float iz = fd(1.0f, z);
    const float J[6] = {fm(cam.fx, iz), 0.0f, fm(-fm(cam.fx, x), fm(iz, iz)),
                        0.0f, fm(cam.fy, iz), fm(-fm(cam.fy, y), fm(iz, iz))};
    float T[6], U[6];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int j = 0; j < 3; j++) T[3 * a + j] = dot3(J[3 * a], R[j], J[3 * a + 1], R[3 + j], J[3 * a + 2], R[6 + j]);
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int j = 0; j < 3; j++) U[3 * a + j] = dot3(T[3 * a], S[j], T[3 * a + 1], S[3 + j], T[3 * a + 2], S[6 + j]);
    const float c00 = dot3(U[0], T[0], U[1], T[1], U[2], T[2]);
    const float c01 = dot3(U[0], T[3], U[1], T[4], U[2], T[5]);
    const float c11 = dot3(U[3], T[3], U[4], T[4], U[5], T[5]);
    const float A = fa(c00, 0.3f), B = c01, Cc = fa(c11, 0.3f);
    const float det = fs(fm(A, Cc), fm(B, B));
    if (det > 0.0f) {
      const float mid = fm(0.5f, fa(A, Cc));
      const float disc = fs(fm(mid, mid), det);
      const float lam = fa(mid, __fsqrt_rn(disc > 0.1f ? disc : 0.1f));
      const float rad = ceilf(fm(3.0f, __fsqrt_rn(lam)));
      const float u = fa(fm(cam.fx, fd(x, z)), cam.cx), v = fa(fm(cam.fy, fd(y, z)), cam.cy);
      const float tx = (float)cam.tiles_x, ty = (float)cam.tiles_y;
      const float fx0 = floorf(fd(fs(u, rad), 16.0f)), fx1 = fa(floorf(fd(fa(u, rad), 16.0f)), 1.0f);
      const float fy0 = floorf(fd(fs(v, rad), 16.0f)), fy1 = fa(floorf(fd(fa(v, rad), 16.0f)), 1.0f);
      const int x0 = fx0 < 0.0f ? 0 : (fx0 > tx ? cam.tiles_x : (int)fx0);
      const int x1 = fx1 < 0.0f ? 0 : (fx1 > tx ? cam.tiles_x : (int)fx1);
      const int y0 = fy0 < 0.0f ? 0 : (fy0 > ty ? cam.tiles_y : (int)fy0);
      const int y1 = fy1 < 0.0f ? 0 : (fy1 > ty ? cam.tiles_y : (int)fy1);
      if (x1 > x0 && y1 > y0) {
        cnt = (uint32_t)((x1 - x0) * (y1 - y0));
        // exp(-(ca dx^2 + 2 cb dx dy + cc dy^2) / 2) = exp2(k0 dx^2 + k1 dx dy + k2 dy^2)
        const float L = 1.4426950408889634f;  // log2(e)
        const float ca = Cc / det, cb = -B / det, cc = A / det;
        const float mu = 1.0f / (1.0f + expf(-lg));  // Eq. sigmoid
        rec[3 * i] = make_float4(u, v, mu, z);
        rec[3 * i + 1] = make_float4(-0.5f * L * ca, -L * cb, -0.5f * L * cc, 0.0f);
        rec[3 * i + 2] = make_float4(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], 0.0f);
        rect[i] = make_int4(x0, y0, x1, y1);
      }
    }
  }
  return cnt;
}

// Splat setup from float geometry in original order.
__global__ void k_splat_setup(int64_t n, const float* __restrict__ pos, const float* __restrict__ scale,
                              const float4* __restrict__ rot, const float* __restrict__ logit,
                              const float* __restrict__ rgb, CamDev cam, float4* __restrict__ rec,
                              int4* __restrict__ rect, uint32_t* __restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float s3[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
    count[i] = splat_one(i, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], s3, rot[i], logit[i], rgb, cam, rec, rect);
  }
}

// Splat setup from the geometry streams, for the slots of the listed groups (the kept chunks');
// counts of the other Gaussians stay 0.
__global__ void k_splat_setup_coded(const int32_t* __restrict__ glist, int64_t n_list, const int32_t* __restrict__ perm,
                                    int64_t n, GeomStreams G, int64_t chunk_slots, const float* __restrict__ rgb,
                                    CamDev cam, float4* __restrict__ rec, int4* __restrict__ rect,
                                    uint32_t* __restrict__ count) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_list * 16; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = glist[v >> 4];
    if (g < 0) continue;
    const int64_t s = (int64_t)g * 16 + (v & 15);
    const int32_t o = perm[s];
    if (o < 0 || o >= n) continue;  // padding (a slot order entry outside [0, n) is skipped too)
    float3 p, sc;
    float4 q;
    float t;
    geom_decode(G, s, chunk_slots, p, sc, q, t);
    const float s3[3] = {sc.x, sc.y, sc.z};
    count[o] = splat_one(o, p.x, p.y, p.z, s3, q, t, rgb, cam, rec, rect);
  }
}

// Decoded centres of the listed groups' Gaussians, in original order (the colour pass's SH
// direction f - p uses them).
__global__ void k_decode_positions(const int32_t* __restrict__ glist, int64_t n_list, const int32_t* __restrict__ perm,
                                   int64_t n, GeomStreams G, int64_t chunk_slots, float* __restrict__ pos) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_list * 16; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = glist[v >> 4];
    if (g < 0) continue;
    const int64_t s = (int64_t)g * 16 + (v & 15);
    const int32_t o = perm[s];
    if (o < 0 || o >= n) continue;
    float3 p, sc;
    float4 q;
    float t;
    geom_decode(G, s, chunk_slots, p, sc, q, t);
    pos[3 * (int64_t)o] = p.x;
    pos[3 * (int64_t)o + 1] = p.y;
    pos[3 * (int64_t)o + 2] = p.z;
  }
}

// The hierarchy's view test: a chunk is kept unless its box of centres, grown by 6 times its
// largest scale, lies entirely at camera depth <= near_z / 2, or entirely in front of the camera
// and more than 64 pixels beyond one image side.
__global__ void k_chunk_visible(int64_t nc, const gsc_chunk* __restrict__ chunk, CamDev cam,
                                uint32_t* __restrict__ vis) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const gsc_chunk e = chunk[c];
    const float g = fm(6.0f, e.max_scale);
    const float* R = cam.R;
    const float hz = fm(0.5f, cam.near_z), W = (float)cam.width, H = (float)cam.height;
    bool behind = true, front = true, left = true, right = true, top = true, bottom = true;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const float cx = (k & 1) ? fa(e.hi[0], g) : fs(e.lo[0], g);
      const float cy = (k & 2) ? fa(e.hi[1], g) : fs(e.lo[1], g);
      const float cz = (k & 4) ? fa(e.hi[2], g) : fs(e.lo[2], g);
      const float x = fa(dot3(R[0], cx, R[1], cy, R[2], cz), cam.t[0]);
      const float y = fa(dot3(R[3], cx, R[4], cy, R[5], cz), cam.t[1]);
      const float z = fa(dot3(R[6], cx, R[7], cy, R[8], cz), cam.t[2]);
      if (z > hz) behind = false;
      if (!(z > hz)) { front = false; continue; }
      const float u = fa(fm(cam.fx, fd(x, z)), cam.cx), v = fa(fm(cam.fy, fd(y, z)), cam.cy);
      if (!(u < -64.0f)) left = false;
      if (!(u > fa(W, 64.0f))) right = false;
      if (!(v < -64.0f)) top = false;
      if (!(v > fa(H, 64.0f))) bottom = false;
    }
    vis[c] = (behind || (front && (left || right || top || bottom))) ? 0u : 1u;
  }
}

// The kept chunks' groups, chunk after chunk (gpc groups per chunk). Only the last chunk can be
// short, and it comes last, so the list is dense: kept * gpc entries less the last chunk's
// missing groups when it is kept.
__global__ void k_chunk_groups(int64_t nc, const uint32_t* __restrict__ vis, const uint32_t* __restrict__ rank,
                               int64_t gpc, int64_t ng, int32_t* __restrict__ glist) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nc * gpc; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / gpc, j = e - c * gpc;
    const int64_t g = c * gpc + j;
    if (vis[c] && g < ng) glist[(int64_t)rank[c] * gpc + j] = (int32_t)g;
  }
}

// Depth keys of the visible Gaussians (culled ones last), for a stable sort that orders them
// nearest first with equal depths in index order; camera depth > near_z > 0, so the float bits
// order like z.
__global__ void k_depth_keys(int64_t n, const float4* __restrict__ rec, const uint32_t* __restrict__ count,
                             uint64_t* __restrict__ dkey, uint32_t* __restrict__ dval) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    dkey[i] = count[i] ? (uint64_t)__float_as_uint(rec[3 * i].w) : 0xFFFFFFFFull;
    dval[i] = (uint32_t)i;
  }
}

// tile counts in depth order
__global__ void k_gather_counts(int64_t n, const uint32_t* __restrict__ dval, const uint32_t* __restrict__ count,
                                uint32_t* __restrict__ out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    out[r] = count[dval[r]];
}

// One tile key per overlapped tile, emitted in depth order: a stable sort by tile then leaves every
// tile's list nearest first (equal depths in index order).
__global__ void k_splat_keys(int64_t n, const uint32_t* __restrict__ dval, const int4* __restrict__ rect,
                             const uint32_t* __restrict__ count_sorted, const uint32_t* __restrict__ offset,
                             int tiles_x, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    if (count_sorted[r] == 0) continue;
    const uint32_t i = dval[r];
    const int4 b = rect[i];
    uint32_t o = offset[r];
    for (int ty = b.y; ty < b.w; ty++)
      for (int tx = b.x; tx < b.z; tx++) {
        keys[o] = (uint64_t)(ty * tiles_x + tx);
        vals[o] = i;
        o++;
      }
  }
}

// ranges[tile] = [first, last + 1) of the tile's entries in the sorted list (empty tiles stay 0)
__global__ void k_tile_ranges(const uint64_t* __restrict__ keys, int64_t P, uint2* __restrict__ ranges) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < P; e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)keys[e];
    if (e == 0 || (uint32_t)keys[e - 1] != t) ranges[t].x = (uint32_t)e;
    if (e == P - 1 || (uint32_t)keys[e + 1] != t) ranges[t].y = (uint32_t)(e + 1);
  }
}

// 2^x on the special-function unit (PTX ex2.approx: relative error about 2^-22; results below
// the normal range flush to zero)
__device__ __forceinline__ float ex2(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Eq. preblend per pixel, the tile's Gaussians nearest first, staged 256 at a time in shared
// memory; 128 threads, each blending two pixels of one tile column (rows y and y + 8) with one
// read of every staged splat (four pixels per thread on 64 threads measured slower: 5.05 against
// 4.33 ms at 1080p). With w = T g, the transmittance update T (1 - mu g) is T - mu w.
#define RTHREADS 128
#define RPIX 2
#define RSTEP 8
#define RBATCH 256
__global__ void __launch_bounds__(RTHREADS) k_render(const uint2* __restrict__ ranges, const uint32_t* __restrict__ vals,
                                                     const float4* __restrict__ rec, int width, int height, int tiles_x,
                                                     float* __restrict__ image, float* __restrict__ trans) {
  __shared__ float4 s0[RBATCH], s1[RBATCH], s2[RBATCH];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * RTILE + (threadIdx.x & (RTILE - 1)), py = ty * RTILE + (threadIdx.x / RTILE);
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 rg = ranges[tile];
  float T[RPIX], r[RPIX], g[RPIX], b[RPIX];
#pragma unroll
  for (int j = 0; j < RPIX; j++) { T[j] = 1.0f; r[j] = 0.0f; g[j] = 0.0f; b[j] = 0.0f; }
  for (uint32_t e0 = rg.x; e0 < rg.y; e0 += RBATCH) {
    __syncthreads();
#pragma unroll
    for (int h = 0; h < RBATCH / RTHREADS; h++) {
      const uint32_t e = e0 + h * RTHREADS + threadIdx.x;
      if (e < rg.y) {
        const uint32_t i = vals[e];
        s0[h * RTHREADS + threadIdx.x] = rec[3 * (int64_t)i];
        s1[h * RTHREADS + threadIdx.x] = rec[3 * (int64_t)i + 1];
        s2[h * RTHREADS + threadIdx.x] = rec[3 * (int64_t)i + 2];
      }
    }
    __syncthreads();
    const int m = (int)min((uint32_t)RBATCH, rg.y - e0);
    for (int k = 0; k < m; k++) {
      const float4 a = s0[k], c = s1[k], col = s2[k];
      const float dx = fx - a.x, dy = fy - a.y;
      const float qx = c.x * dx;  // the exponent is dx (k0 dx + k1 dy) + k2 dy^2
#pragma unroll
      for (int j = 0; j < RPIX; j++) {
        const float d = dy + (float)(RSTEP * j);
        const float q = dx * (qx + c.y * d) + c.z * d * d;
        const float w = T[j] * ex2(q);
        r[j] += w * col.x;
        g[j] += w * col.y;
        b[j] += w * col.z;
        T[j] -= a.z * w;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < RPIX; j++) {
    if (px < width && py + RSTEP * j < height) {
      const int64_t p = (int64_t)(py + RSTEP * j) * width + px;
      image[3 * p] = r[j];
      image[3 * p + 1] = g[j];
      image[3 * p + 2] = b[j];
      if (trans) trans[p] = T[j];
    }
  }
}

int grid_of(int64_t work) {
  int64_t g = ceil_div64(work, 256);
  if (g > gsc_sm_count() * 16) g = gsc_sm_count() * 16;
  return (int)(g < 1 ? 1 : g);
}

bool cam_ok(const gsc_camera* c) {
  if (!c || c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384) return false;
  const float v[4] = {c->fx, c->fy, c->near_z, c->cx};
  if (!(v[0] > 0.0f) || !(v[1] > 0.0f) || !(v[2] > 0.0f) || !isfinite(v[0]) || !isfinite(v[1])) return false;
  for (int k = 0; k < 9; k++) if (!isfinite(c->R[k])) return false;
  for (int k = 0; k < 3; k++) if (!isfinite(c->t[k])) return false;
  return isfinite(c->cx) && isfinite(c->cy) && isfinite(c->near_z);
}

int tile_bits(int64_t tiles) {
  int b = 1;
  while ((1ll << b) < tiles) b++;
  return b;
}

struct RenderWs {
  float* f;
  float* rgb;
  float4* rec;
  int4* rect;
  uint32_t *count, *offset;
  uint64_t* total;
  void* scan_ws;
  uint2* ranges;
  uint64_t* dkey;
  uint32_t *dval, *count_sorted;
  uint32_t *vis, *vrank;
  int32_t* glist;
  float* pos_dec;
  uint64_t* keys;
  uint32_t* vals;
  void* radix_ws;
};

// fixed part first, then the buffers that grow with the number of (Gaussian, tile) pairs
// nc / ng: chunks and groups of the coded path (0 for float geometry)
RenderWs carve_render(void* ws, size_t cap, int64_t n, int64_t tiles, int64_t pairs, int64_t nc, int64_t ng, bool* ok) {
  Carve c{reinterpret_cast<uint8_t*>(ws), 0, cap};
  RenderWs w;
  w.f = c.take<float>(4);
  w.rgb = c.take<float>(3 * n);
  w.rec = c.take<float4>(3 * n);
  w.rect = c.take<int4>(n);
  w.count = c.take<uint32_t>(n);
  w.offset = c.take<uint32_t>(n);
  w.total = c.take<uint64_t>(1);
  w.scan_ws = c.take<uint8_t>((int64_t)scan_ws_bytes(n));
  w.ranges = c.take<uint2>(tiles);
  w.dkey = c.take<uint64_t>(n);
  w.dval = c.take<uint32_t>(n);
  w.count_sorted = c.take<uint32_t>(n);
  w.vis = c.take<uint32_t>(nc);
  w.vrank = c.take<uint32_t>(nc);
  w.glist = c.take<int32_t>(ng);
  w.pos_dec = c.take<float>(ng > 0 ? 3 * n : 0);
  w.keys = c.take<uint64_t>(pairs);
  w.vals = c.take<uint32_t>(pairs);
  w.radix_ws = c.take<uint8_t>((int64_t)radix_ws_bytes(pairs > n ? pairs : n));
  *ok = c.ok();
  return w;
}

size_t render_bytes(int64_t n, int64_t tiles, int64_t pairs, int64_t nc, int64_t ng) {
  size_t b = 0;
  auto add = [&](int64_t bytes) { b = align_up(b, 256) + (size_t)(bytes > 8 ? bytes : 8); };
  add(4 * 4);
  add(4 * 3 * n);
  add(16 * 3 * n);
  add(16 * n);
  add(4 * n);
  add(4 * n);
  add(8);
  add((int64_t)scan_ws_bytes(n));
  add(8 * tiles);
  add(8 * n);
  add(4 * n);
  add(4 * n);
  add(4 * nc);
  add(4 * nc);
  add(4 * ng);
  add(ng > 0 ? 12 * n : 0);
  add(8 * pairs);
  add(4 * pairs);
  add((int64_t)radix_ws_bytes(pairs > n ? pairs : n));
  return align_up(b, 256) + 256;
}

}  // namespace

extern "C" size_t gsc_render_workspace_bytes(int64_t n, const gsc_camera* cam, int64_t max_pairs) {
  if (n < 0 || max_pairs < 0 || !cam_ok(cam)) return 0;
  const int64_t tiles = (int64_t)((cam->width + RTILE - 1) / RTILE) * ((cam->height + RTILE - 1) / RTILE);
  const int64_t ng = (n + 15) / 16;
  // room for the coded path's chunk and group lists too (at most one chunk per group)
  return render_bytes(n, tiles, max_pairs, ng, ng);
}

namespace {

// The shared pipeline: colour (fused decode + SH for the camera centre), splat setup (float geometry,
// or the streams of the kept chunks), depth sort, tile keys, tile sort, ranges, blending.
gsc_status render_run(gsc_ctx* c, const DevTable& T, const uint8_t* d_blocks, const int32_t* d_perm,
                      const float* d_pos, const float* d_scale, const float* d_rot, const float* d_logit,
                      const uint8_t* d_geom, int64_t chunk_slots, const gsc_camera* cam, float* d_image,
                      float* d_trans, int64_t* h_pairs, int64_t* h_chunks, void* d_ws, size_t ws_bytes,
                      cudaStream_t st) {
  const int64_t n = T.n, ng = T.n_groups, ns = ng * 16;
  const bool coded = d_geom != nullptr;
  const int64_t nc = coded ? (ns + chunk_slots - 1) / chunk_slots : 0, gpc = coded ? chunk_slots / 16 : 0;
  CamDev cd;
  memcpy(cd.R, cam->R, sizeof(cd.R));
  memcpy(cd.t, cam->t, sizeof(cd.t));
  cd.fx = cam->fx; cd.fy = cam->fy; cd.cx = cam->cx; cd.cy = cam->cy; cd.near_z = cam->near_z;
  cd.width = cam->width; cd.height = cam->height;
  cd.tiles_x = (cam->width + RTILE - 1) / RTILE;
  cd.tiles_y = (cam->height + RTILE - 1) / RTILE;
  const int64_t tiles = (int64_t)cd.tiles_x * cd.tiles_y;
  bool ok = false;
  RenderWs w = carve_render(d_ws, ws_bytes, n, tiles, 0, coded ? ng : 0, coded ? ng : 0, &ok);
  if (!ok) return GSC_ERR_OOM;
  GscTimed tm(c, T_RENDER, st);
  // camera centre f = -R^T t (the SH direction is f - p), rounded to float once
  float* hp = reinterpret_cast<float*>(c->h_pinned);
  for (int k = 0; k < 3; k++) {
    const double v = ((double)cam->R[k] * cam->t[0] + (double)cam->R[3 + k] * cam->t[1]) + (double)cam->R[6 + k] * cam->t[2];
    hp[k] = (float)(-v);
  }
  uint64_t* hcount = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(c->h_pinned) + 64);
  GSC_CUDA(cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * (size_t)tiles, st));
  uint64_t pairs = 0, kept = 0;
  if (n > 0) {
    GSC_CUDA(cudaMemcpyAsync(w.f, hp, 3 * sizeof(float), cudaMemcpyHostToDevice, st));
    if (coded) {
      // the hierarchy first: kept chunks, then their groups' colours and splats only
      const GeomStreams G = geom_streams(const_cast<uint8_t*>(d_geom), ns, chunk_slots);
      gsc_count_launch();
      k_chunk_visible<<<grid_of(nc), 256, 0, st>>>(nc, G.chunk, cd, w.vis);
      GSC_CUDA(cudaGetLastError());
      GSC_CUDA(scan_exclusive<uint32_t>(w.vis, w.vrank, nc, w.total, w.scan_ws, st));
      gsc_count_launch();
      k_chunk_groups<<<grid_of(nc * gpc), 256, 0, st>>>(nc, w.vis, w.vrank, gpc, ng, w.glist);
      GSC_CUDA(cudaGetLastError());
      uint32_t* hlast = reinterpret_cast<uint32_t*>(hcount + 1);
      GSC_CUDA(cudaMemcpyAsync(hcount, w.total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      GSC_CUDA(cudaMemcpyAsync(hlast, w.vis + (nc - 1), sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      GSC_CUDA(cudaStreamSynchronize(st));
      kept = *hcount;
      const int64_t n_list = (int64_t)kept * gpc - (*hlast ? nc * gpc - ng : 0);
      GSC_CUDA(cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * (size_t)n, st));
      if (n_list > 0) {
        gsc_count_launch();
        k_decode_positions<<<grid_of(n_list * 16), 256, 0, st>>>(w.glist, n_list, d_perm, n, G, chunk_slots,
                                                                  w.pos_dec);
        GSC_CUDA(cudaGetLastError());
        GSC_CUDA(launch_decode_eval(T, d_blocks, d_perm, nullptr, w.pos_dec, w.f, 1, GSC_OUT_GAUSS_MAJOR, w.rgb,
                                    c->sm_count, st, w.glist, n_list));
        gsc_count_launch();
        k_splat_setup_coded<<<grid_of(n_list * 16), 256, 0, st>>>(w.glist, n_list, d_perm, n, G, chunk_slots, w.rgb,
                                                                   cd, w.rec, w.rect, w.count);
        GSC_CUDA(cudaGetLastError());
      }
    } else {
      GSC_CUDA(launch_decode_eval(T, d_blocks, d_perm, nullptr, d_pos, w.f, 1, GSC_OUT_GAUSS_MAJOR, w.rgb, c->sm_count, st));
      gsc_count_launch();
      k_splat_setup<<<grid_of(n), 256, 0, st>>>(n, d_pos, d_scale, reinterpret_cast<const float4*>(d_rot), d_logit,
                                               w.rgb, cd, w.rec, w.rect, w.count);
      GSC_CUDA(cudaGetLastError());
    }
    // visible Gaussians nearest first (stable: equal depths in index order), their counts in that order
    gsc_count_launch();
    k_depth_keys<<<grid_of(n), 256, 0, st>>>(n, w.rec, w.count, w.dkey, w.dval);
    GSC_CUDA(cudaGetLastError());
    GSC_CUDA(radix_sort_pairs(w.dkey, w.dval, n, 32, w.radix_ws, st));
    gsc_count_launch();
    k_gather_counts<<<grid_of(n), 256, 0, st>>>(n, w.dval, w.count, w.count_sorted);
    GSC_CUDA(cudaGetLastError());
    GSC_CUDA(scan_exclusive<uint32_t>(w.count_sorted, w.offset, n, w.total, w.scan_ws, st));
    GSC_CUDA(cudaMemcpyAsync(hcount, w.total, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    GSC_CUDA(cudaStreamSynchronize(st));
    pairs = *hcount;
  }
  if (h_pairs) *h_pairs = (int64_t)pairs;
  if (h_chunks) *h_chunks = (int64_t)kept;
  if (pairs > 0xFFFFFFF0ull) return GSC_ERR_OOM;
  w = carve_render(d_ws, ws_bytes, n, tiles, (int64_t)pairs, coded ? ng : 0, coded ? ng : 0, &ok);
  if (!ok) return GSC_ERR_OOM;
  if (pairs > 0) {
    gsc_count_launch();
    k_splat_keys<<<grid_of(n), 256, 0, st>>>(n, w.dval, w.rect, w.count_sorted, w.offset, cd.tiles_x, w.keys,
                                             w.vals);
    GSC_CUDA(cudaGetLastError());
    GSC_CUDA(radix_sort_pairs(w.keys, w.vals, (int64_t)pairs, tile_bits(tiles), w.radix_ws, st));
    gsc_count_launch();
    k_tile_ranges<<<grid_of((int64_t)pairs), 256, 0, st>>>(w.keys, (int64_t)pairs, w.ranges);
    GSC_CUDA(cudaGetLastError());
  }
  GscTimed tb(c, T_BLEND, st);
  gsc_count_launch();
  k_render<<<(int)tiles, RTHREADS, 0, st>>>(w.ranges, w.vals, w.rec, cam->width, cam->height, cd.tiles_x, d_image,
                                           d_trans);
  GSC_CUDA(cudaGetLastError());
  return GSC_OK;
}

}  // namespace

extern "C" gsc_status gsc_render(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                 const int32_t* d_perm, const float* d_pos, const float* d_scale, const float* d_rot,
                                 const float* d_logit, const gsc_camera* cam, float* d_image, float* d_trans,
                                 int64_t* h_pairs, void* d_ws, size_t ws_bytes, void* stream) {
  GscRange gsc_range_("gsc_render");
  if (!c || !cam_ok(cam)) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (!d_image || (T.n > 0 && (!d_blocks || !d_perm || !d_pos || !d_scale || !d_rot || !d_logit || !d_ws)))
    return GSC_ERR_INVALID_ARG;
  auto al = [](const void* p, uintptr_t a) { return ((uintptr_t)p % a) == 0; };
  if (!al(d_blocks, 8) || !al(d_rot, 16) || !al(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  return render_run(c, T, d_blocks, d_perm, d_pos, d_scale, d_rot, d_logit, nullptr, 0, cam, d_image, d_trans, h_pairs,
                    nullptr, d_ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" gsc_status gsc_render_coded(gsc_ctx* c, const gsc_stream_table* table, const uint8_t* d_blocks,
                                       const int32_t* d_perm, const uint8_t* d_geom, int64_t chunk_slots,
                                       const gsc_camera* cam, float* d_image, float* d_trans, int64_t* h_pairs,
                                       int64_t* h_chunks, void* d_ws, size_t ws_bytes, void* stream) {
  GscRange gsc_range_("gsc_render_coded");
  if (!c || !cam_ok(cam) || chunk_slots < 16 || chunk_slots % 16) return GSC_ERR_INVALID_ARG;
  DevTable T;
  gsc_status s = make_dev_table(table, &T);
  if (s != GSC_OK) return s;
  if (!d_image || (T.n > 0 && (!d_blocks || !d_perm || !d_geom || !d_ws))) return GSC_ERR_INVALID_ARG;
  auto al = [](const void* p, uintptr_t a) { return ((uintptr_t)p % a) == 0; };
  if (!al(d_blocks, 8) || !al(d_geom, 256) || !al(d_ws, 256)) return GSC_ERR_INVALID_ARG;
  GSC_CUDA(cudaSetDevice(c->device));
  // the colour pass's SH direction uses the decoded centres
  return render_run(c, T, d_blocks, d_perm, nullptr, nullptr, nullptr, nullptr, d_geom, chunk_slots, cam, d_image,
                    d_trans, h_pairs, h_chunks, d_ws, ws_bytes, (cudaStream_t)stream);
}
