// Headless rasterisation (the paper's rasterisation pass, Sec. "Experimental
// results", without a graphics API): triangles -> a fragment buffer holding,
// per pixel, the nearest triangle's id and perspective-correct barycentrics;
// then per-pixel shading by interpolating per-vertex radiance.
//
// Coverage and depth decisions are made in float32 with a fixed operation
// order and no fused multiply-add (the _rn intrinsics), so they are a pure
// function of the inputs: the pixel centre (px + 1/2, py + 1/2) is covered when
// the three edge functions, oriented to a positive area, are > 0, or = 0 on an
// edge whose direction (dx, dy) has dy > 0, or dy = 0 and dx < 0 (a shared
// edge is seen in opposite directions by its two triangles, so it is covered
// once).  The nearest depth wins through a 64-bit atomicMin on (depth bits,
// triangle id): depth >= 0 floats order like their bit patterns, and equal
// depths keep the lower id.
#include "common.cuh"

namespace hs {

__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by, float px, float py) {
  return __fsub_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(py, ay)), __fmul_rn(__fsub_rn(by, ay), __fsub_rn(px, ax)));
}

// clip = M [x y z 1] (row-major), ndc = clip / w, screen x = (ndc_x + 1) / 2 * width,
// y = (1 - ndc_y) / 2 * height; out = (x, y, ndc z, w)
__global__ void k_raster_project(int V, const float* __restrict__ pos, const float* __restrict__ M, int width,
                                 int height, float4* __restrict__ sv) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float x = pos[3 * v], y = pos[3 * v + 1], z = pos[3 * v + 2];
  float c[4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
    c[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(M[4 * r], x), __fmul_rn(M[4 * r + 1], y)), __fmul_rn(M[4 * r + 2], z)),
                     M[4 * r + 3]);
  const float nx = __fdiv_rn(c[0], c[3]), ny = __fdiv_rn(c[1], c[3]), nz = __fdiv_rn(c[2], c[3]);
  sv[v] = make_float4(__fmul_rn(__fmul_rn(__fadd_rn(nx, 1.0f), 0.5f), (float)width),
                      __fmul_rn(__fmul_rn(__fsub_rn(1.0f, ny), 0.5f), (float)height), nz, c[3]);
}

__global__ void k_raster_clear(long long n, unsigned long long* __restrict__ zbuf) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) zbuf[p] = ~0ull;
}

__device__ __forceinline__ bool owns(float ax, float ay, float bx, float by) {
  const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay);
  return dy > 0.0f || (dy == 0.0f && dx < 0.0f);
}

// One thread per triangle: its pixel bounding box, the edge tests and the
// depth test of every pixel centre in it.
__global__ void k_raster_tris(int V, int T, const int32_t* __restrict__ tris, const float4* __restrict__ sv,
                              int width, int height, unsigned long long* __restrict__ zbuf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int i0 = tris[3 * t], i1 = tris[3 * t + 1], i2 = tris[3 * t + 2];
  if (i0 < 0 || i0 >= V || i1 < 0 || i1 >= V || i2 < 0 || i2 >= V) return;   // invalid triangles are dropped
  float4 a = sv[i0], b = sv[i1], c = sv[i2];
  if (!(a.w > 1e-6f && b.w > 1e-6f && c.w > 1e-6f)) return;                    // no near-plane clipping
  float area = edge_fn(a.x, a.y, b.x, b.y, c.x, c.y);
  if (!isfinite(area) || area == 0.0f) return;
  if (area < 0.0f) {
    const float4 tmp = b;
    b = c;
    c = tmp;
    area = -area;
  }
  const float fx0 = fmaxf(floorf(fminf(fminf(a.x, b.x), c.x)), 0.0f);
  const float fx1 = fminf(ceilf(fmaxf(fmaxf(a.x, b.x), c.x)), (float)(width - 1));
  const float fy0 = fmaxf(floorf(fminf(fminf(a.y, b.y), c.y)), 0.0f);
  const float fy1 = fminf(ceilf(fmaxf(fmaxf(a.y, b.y), c.y)), (float)(height - 1));
  if (!(fx0 <= fx1 && fy0 <= fy1)) return;
  const bool o0 = owns(b.x, b.y, c.x, c.y), o1 = owns(c.x, c.y, a.x, a.y), o2 = owns(a.x, a.y, b.x, b.y);
  const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
  for (int py = y0; py <= y1; ++py) {
    const float pyc = (float)py + 0.5f;
    for (int px = x0; px <= x1; ++px) {
      const float pxc = (float)px + 0.5f;
      const float e0 = edge_fn(b.x, b.y, c.x, c.y, pxc, pyc);
      const float e1 = edge_fn(c.x, c.y, a.x, a.y, pxc, pyc);
      const float e2 = edge_fn(a.x, a.y, b.x, b.y, pxc, pyc);
      const bool in = (e0 > 0.0f || (e0 == 0.0f && o0)) && (e1 > 0.0f || (e1 == 0.0f && o1)) &&
                      (e2 > 0.0f || (e2 == 0.0f && o2));
      if (!in) continue;
      const float zi = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(e0, a.z), __fmul_rn(e1, b.z)), __fmul_rn(e2, c.z)), area);
      const float depth = __fmul_rn(__fadd_rn(zi, 1.0f), 0.5f);
      if (!(depth >= 0.0f && depth <= 1.0f)) continue;
      const unsigned long long key = ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned)t;
      atomicMin(zbuf + (long long)py * width + px, key);
    }
  }
}

// One thread per pixel: the winner's id and perspective-correct barycentrics
// (screen weights of the triangle's own vertex order divided by each w).
__global__ void k_raster_resolve(int width, int height, const unsigned long long* __restrict__ zbuf,
                                 const int32_t* __restrict__ tris, const float4* __restrict__ sv,
                                 int32_t* __restrict__ tri_id, float2* __restrict__ bary) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)width * height) return;
  const unsigned long long key = zbuf[p];
  if (key == ~0ull) {
    tri_id[p] = -1;
    bary[p] = make_float2(0.0f, 0.0f);
    return;
  }
  const int t = (int)(key & 0xffffffffull);
  const int px = (int)(p % width), py = (int)(p / width);
  const float pxc = (float)px + 0.5f, pyc = (float)py + 0.5f;
  const float4 a = sv[tris[3 * t]], b = sv[tris[3 * t + 1]], c = sv[tris[3 * t + 2]];
  const float a0 = edge_fn(b.x, b.y, c.x, c.y, pxc, pyc) / a.w;
  const float a1 = edge_fn(c.x, c.y, a.x, a.y, pxc, pyc) / b.w;
  const float a2 = edge_fn(a.x, a.y, b.x, b.y, pxc, pyc) / c.w;
  const float inv = 1.0f / (a0 + a1 + a2);
  tri_id[p] = t;
  bary[p] = make_float2(a1 * inv, a2 * inv);
}

// One thread per pixel: radiance interpolated from the triangle's vertices,
// the background where nothing is hit (or the id is not a valid triangle).
__global__ void k_shade_pixels(long long P, int C, int V, int T, const int32_t* __restrict__ tri_id,
                               const float2* __restrict__ bary, const int32_t* __restrict__ tris,
                               const float* __restrict__ rad, const float* __restrict__ bg, float* __restrict__ img) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int t = tri_id[p];
  float* o = img + p * C;
  int i0 = -1, i1 = -1, i2 = -1;
  if (t >= 0 && t < T) {
    i0 = tris[3 * t];
    i1 = tris[3 * t + 1];
    i2 = tris[3 * t + 2];
  }
  if (i0 < 0 || i0 >= V || i1 < 0 || i1 >= V || i2 < 0 || i2 >= V) {
    for (int ch = 0; ch < C; ++ch) o[ch] = bg[ch];
    return;
  }
  const float2 w = bary[p];
  const float w0 = 1.0f - w.x - w.y;
  for (int ch = 0; ch < C; ++ch)
    o[ch] = w0 * rad[(long long)i0 * C + ch] + w.x * rad[(long long)i1 * C + ch] + w.y * rad[(long long)i2 * C + ch];
}

haar_status_t launch_rasterize(int V, const float* pos, int T, const int32_t* tris, const float* M, int width,
                               int height, float* screen, unsigned long long* zbuf, int32_t* tri_id, float* bary,
                               cudaStream_t st) {
  float4* sv = reinterpret_cast<float4*>(screen);
  const long long P = (long long)width * height;
  k_raster_clear<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, zbuf);
  if (V > 0) k_raster_project<<<(V + 255) / 256, 256, 0, st>>>(V, pos, M, width, height, sv);
  if (T > 0) k_raster_tris<<<(T + 127) / 128, 128, 0, st>>>(V, T, tris, sv, width, height, zbuf);
  k_raster_resolve<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(width, height, zbuf, tris, sv, tri_id,
                                                                reinterpret_cast<float2*>(bary));
  return cuda_check(cudaGetLastError(), "rasterize launch");
}

haar_status_t launch_shade_pixels(int width, int height, int C, int V, int T, const int32_t* tri_id,
                                  const float* bary, const int32_t* tris, const float* rad, const float* bg,
                                  float* img, cudaStream_t st) {
  const long long P = (long long)width * height;
  k_shade_pixels<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(P, C, V, T, tri_id,
                                                             reinterpret_cast<const float2*>(bary), tris, rad, bg,
                                                             img);
  return cuda_check(cudaGetLastError(), "k_shade_pixels launch");
}

}  // namespace hs
