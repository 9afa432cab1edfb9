// Haar-domain phase shift on sm_103a: per-launch set-up (FP64 shift
// parameters, pixel synthesis), the tile-fused resample + forward-Haar
// kernel with the coarse levels finished by the last tile of each shift,
// and the batched forward / inverse transforms.
//
// The operator is the paper's phase shift of a lat-long map's Haar
// coefficients (Sec. "Rotating Haar", Eq. tRot/theta/phi/compfunc):
//   c' = Haar( resample( Haar^-1 c ) ).
// Per launch the map is synthesised once (C*H*W floats, L2-resident) and
// every (shift, 64x64 output tile) CTA resamples its tile, runs levels 1..6
// of the forward transform in shared memory and writes those coefficients
// straight to their canonical positions; the tile means (the level-6
// scaling image) go to the workspace and the last CTA of each shift
// transforms them into the coarse levels (Sec. "Algorithmic optimization":
// every level follows from the previous one, O(N) in total).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"
#include "rotcoord.cuh"
#include "tc.cuh"

namespace hs {

constexpr int kThreads = 256;
constexpr int kRotChannels = 3;   // channels resampled together by the rotation kernel (RGB)

enum { KIND_TRANSLATE = 0, KIND_ROTATE = 1, KIND_COPY = 2 };

struct ShiftArgs {
  Geometry g;
  int K;                  // coefficients written per (s, c)
  long long st_s, st_c, st_k;
  long long plane;        // hi -> lo plane offset (BF16_HILO)
  void* out;
  const float* pix;       // source pixels [C][H][W] (or maps [batch][H][W] for KIND_COPY)
  const float* cin;       // input coefficients [C][cin_stride] (signed-permutation copies)
  long long cin_stride;
  const ShiftParam* prm;  // [S] or null
  float* means;           // [S][C][n_tiles] (null: means go to out[..., 0:n_tiles])
  unsigned* counters;     // [S] (null: no in-kernel coarse pass)
  const float4* rows;     // rotations: [H] (sin theta_i hi, lo, cos theta_i hi, lo)
  const float4* rtab;     // rotations: per-rotation tables, rt_stride float4 apart
  long long rt_stride;
  int tab_off;            // rotations, tables in shared memory: their offset in floats
  int tail_off = 0;       // translation batch kernel: the tail's offset in floats (tr8_tail_floats)
  float scale;
  float u_scale, v_scale; // H/pi, W/(2 pi)
  const float* pixE = nullptr;   // translation batches: the extended map (see haar_shift_plan_s::pixE)
  int HE = 0, WE = 0;
  int* status = nullptr;         // device status word (bounded waits)
};

// The two row taps of a rotated sample as texel offsets into the interleaved
// rotation map (each texel holds columns c and c + 1): rows beyond a pole are
// the mirrored row half a turn away (SPHERE) or wrap (TORUS).
__device__ __forceinline__ void rot_taps(const RotSrc& o, int H, int W, int boundary, int& t0, int& t1) {
  int r0 = o.r, r1 = o.r + 1, h0 = 0, h1 = 0;
  if (boundary == HAAR_BOUNDARY_TORUS) {
    r0 &= H - 1;
    r1 &= H - 1;
  } else {
    if (r0 < 0) { r0 = 0; h0 = W >> 1; }
    if (r1 >= H) { r1 = H - 1; h1 = W >> 1; }
  }
  t0 = r0 * W + ((o.c + h0) & (W - 1));
  t1 = r1 * W + ((o.c + h1) & (W - 1));
}

// One 32-byte texel of the interleaved rotation map in one load (32-byte
// aligned): v[2c], v[2c+1] = channel c at columns j and j+1.
__device__ __forceinline__ void ld_texel(const float4* p, float (&v)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}

// Bilinear value of channel ci (0..2) of a texel pair (rows t0, t1).
__device__ __forceinline__ float rot_lerp(float a0, float a1, float b0, float b1, float fu, float fv) {
  const float top = fmaf(fv, a1 - a0, a0), bot = fmaf(fv, b1 - b0, b0);
  return fmaf(fu, bot - top, top);
}

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void ext_index(int& i, int& j, int H, int W, int boundary) {
  if (boundary == HAAR_BOUNDARY_TORUS) {
    i %= H;
    if (i < 0) i += H;
  } else {
#pragma unroll 1
    for (int it = 0; it < 8 && (i < 0 || i >= H); ++it) {
      i = (i < 0) ? -1 - i : 2 * H - 1 - i;
      j += W >> 1;
    }
  }
  j %= W;
  if (j < 0) j += W;
}

template <int OUT>
__device__ __forceinline__ void put(const ShiftArgs& a, int s, int c, int k, float v) {
  if (k >= a.K) return;
  long long idx = (long long)s * a.st_s + (long long)c * a.st_c + (long long)k * a.st_k;
  if (OUT == HAAR_OUT_F32) {
    reinterpret_cast<float*>(a.out)[idx] = v * a.scale;
  } else if (OUT == HAAR_OUT_BF16_HILO) {
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    reinterpret_cast<__nv_bfloat16*>(a.out)[idx] = hi;
    reinterpret_cast<__nv_bfloat16*>(a.out)[a.plane + idx] = lo;
  } else {
    reinterpret_cast<__half*>(a.out)[idx] = __float2half_rn(v);
  }
}

// Closed-form source of a block moved by a block-aligned integer shift: the
// level-l coefficients are a signed permutation of the input's (a block
// mirrored across a pole moves half a turn and its V, D change sign).
__device__ float perm_value(const ShiftArgs& a, const ShiftParam& p, int c, int lvl, int band,
                            int r, int col) {
  const Geometry& g = a.g;
  const int l = lvl > g.n ? g.n : lvl;
  const int B = 1 << l;
  const int rows = lvl > g.n ? 1 : (g.H >> l);
  const int cols = lvl > g.n ? g.q : (g.W >> l);
  int rs = r - p.ky / B, cs = col - p.kx / B;
  bool flip = false;
  if (g.boundary == HAAR_BOUNDARY_TORUS) {
    rs %= rows;
    if (rs < 0) rs += rows;
  } else {
#pragma unroll 1
    for (int it = 0; it < 8 && (rs < 0 || rs >= rows); ++it) {
      rs = rs < 0 ? -1 - rs : 2 * rows - 1 - rs;
      cs += (g.W >> 1) / B;
      flip = !flip;
    }
  }
  cs %= cols;
  if (cs < 0) cs += cols;
  const float* src = a.cin + (long long)c * a.cin_stride;
  if (lvl > g.n) return __ldg(src + cs);
  const long long gl = (long long)g.q << (2 * (g.n - l));
  float v = __ldg(src + gl * (1 + band) + (long long)rs * cols + cs);
  return (flip && band != 0) ? -v : v;
}

template <int OUT>
__device__ __forceinline__ void store_at(const ShiftArgs& a, long long idx, float v) {
  if (OUT == HAAR_OUT_F32) {
    reinterpret_cast<float*>(a.out)[idx] = v * a.scale;
  } else if (OUT == HAAR_OUT_BF16_HILO) {
    __nv_bfloat16 hi = __float2bfloat16_rn(v);
    __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    reinterpret_cast<__nv_bfloat16*>(a.out)[idx] = hi;
    reinterpret_cast<__nv_bfloat16*>(a.out)[a.plane + idx] = lo;
  } else {
    reinterpret_cast<__half*>(a.out)[idx] = __float2half_rn(v);
  }
}

// Detail coefficients (H, V, D) of block (r, col) of level lvl; levels whose
// block side divides an integer shift are replaced by the signed permutation
// of the input (bit-exact copies).
template <int OUT>
__device__ __forceinline__ void emit(const ShiftArgs& a, const ShiftParam* p, int s, int c, int lvl,
                                     int r, int col, float hv, float vv, float dv) {
  const Geometry& g = a.g;
  const int gl = g.q << (2 * (g.n - lvl));
  if (gl >= a.K) return;                      // whole level truncated away
  const int k0 = gl + r * (g.W >> lvl) + col;
  if (p != nullptr && ((p->perm_mask >> lvl) & 1u)) {
    hv = perm_value(a, *p, c, lvl, 0, r, col);
    vv = perm_value(a, *p, c, lvl, 1, r, col);
    dv = perm_value(a, *p, c, lvl, 2, r, col);
  }
  const long long bsc = (long long)s * a.st_s + (long long)c * a.st_c;
  const long long sk = a.st_k;
  if (4 * gl <= a.K) {
    store_at<OUT>(a, bsc + k0 * sk, hv);
    store_at<OUT>(a, bsc + (k0 + gl) * sk, vv);
    store_at<OUT>(a, bsc + (k0 + 2 * gl) * sk, dv);
  } else {
    if (k0 < a.K) store_at<OUT>(a, bsc + k0 * sk, hv);
    if (k0 + gl < a.K) store_at<OUT>(a, bsc + (k0 + gl) * sk, vv);
    if (k0 + 2 * gl < a.K) store_at<OUT>(a, bsc + (k0 + 2 * gl) * sk, dv);
  }
}

// Levels lvl0+1 and lvl0+2 of one 4 x 4 block x (row-major) whose element
// (0, 0) sits at level-lvl0 grid position (gr0 + 4 by, gc0 + 4 bx): writes the
// detail coefficients and returns the block's scaling value.
template <int OUT>
__device__ __forceinline__ float block4(const ShiftArgs& a, const ShiftParam* p, int s, int c, const float* x,
                                        int lvl0, int gr0, int gc0, int by, int bx) {
  float A1[4];
#pragma unroll
  for (int sa = 0; sa < 2; ++sa) {
#pragma unroll
    for (int sc = 0; sc < 2; ++sc) {
      const float ea = x[(2 * sa) * 4 + 2 * sc], eb = x[(2 * sa) * 4 + 2 * sc + 1];
      const float ec = x[(2 * sa + 1) * 4 + 2 * sc], ed = x[(2 * sa + 1) * 4 + 2 * sc + 1];
      A1[2 * sa + sc] = 0.5f * ((ea + eb) + (ec + ed));
      emit<OUT>(a, p, s, c, lvl0 + 1, (gr0 >> 1) + 2 * by + sa, (gc0 >> 1) + 2 * bx + sc,
                0.5f * ((eb + ed) - (ea + ec)), 0.5f * ((ec + ed) - (ea + eb)), 0.5f * ((ea + ed) - (eb + ec)));
    }
  }
  const float ea = A1[0], eb = A1[1], ec = A1[2], ed = A1[3];
  emit<OUT>(a, p, s, c, lvl0 + 2, (gr0 >> 2) + by, (gc0 >> 2) + bx, 0.5f * ((eb + ed) - (ea + ec)),
            0.5f * ((ec + ed) - (ea + eb)), 0.5f * ((ea + ed) - (eb + ec)));
  return 0.5f * ((ea + eb) + (ec + ed));
}

// One pass of the forward transform over a rows x cols image in shared
// memory (row pitch = cols): every thread takes a block of side sb (4: two
// levels, 2: one level), writes the detail coefficients of levels lvl0+1
// (and lvl0+2) and the block's scaling value to dst (pitch cols/sb).
// (gr0, gc0) = level-lvl0 grid position of the image's element (0, 0).
template <int OUT>
__device__ void haar_pass(const ShiftArgs& a, const ShiftParam* p, int s, int c, const float* src,
                          float* dst, int rows, int cols, int lvl0, int sb, int gr0, int gc0,
                          int tid, int nthr) {
  const int nbr = rows / sb, nbc = cols / sb;
  const int sh = __ffs(nbc) - 1;              // nbc is a power of two
  for (int b = tid; b < nbr * nbc; b += nthr) {
    const int by = b >> sh, bx = b & (nbc - 1);
    if (sb == 4) {
      float x[16];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float4 t = *reinterpret_cast<const float4*>(src + (4 * by + r) * cols + 4 * bx);
        x[4 * r + 0] = t.x; x[4 * r + 1] = t.y; x[4 * r + 2] = t.z; x[4 * r + 3] = t.w;
      }
      dst[by * nbc + bx] = block4<OUT>(a, p, s, c, x, lvl0, gr0, gc0, by, bx);
    } else {
      const float ea = src[(2 * by) * cols + 2 * bx], eb = src[(2 * by) * cols + 2 * bx + 1];
      const float ec = src[(2 * by + 1) * cols + 2 * bx], ed = src[(2 * by + 1) * cols + 2 * bx + 1];
      emit<OUT>(a, p, s, c, lvl0 + 1, (gr0 >> 1) + by, (gc0 >> 1) + bx,
                0.5f * ((eb + ed) - (ea + ec)), 0.5f * ((ec + ed) - (ea + eb)),
                0.5f * ((ea + ed) - (eb + ec)));
      dst[by * nbc + bx] = 0.5f * ((ea + eb) + (ec + ed));
    }
  }
}

// Levels 1..Lt of one T x T tile held in buf0 (buf1 is scratch of (T/4)^2
// floats).  Returns (to thread 0) the tile's scaling value.
template <int OUT>
__device__ float tile_levels(const ShiftArgs& a, const ShiftParam* p, int s, int c, float* buf0,
                             float* buf1, int tr, int tc) {
  const int T = a.g.T;
  int side = T, lvl = 0;
  float* src = buf0;
  float* dst = buf1;
  while (lvl < a.g.Lt) {
    const int sb = (a.g.Lt - lvl >= 2) ? 4 : 2;
    __syncthreads();
    haar_pass<OUT>(a, p, s, c, src, dst, side, side, lvl, sb, (tr * T) >> lvl, (tc * T) >> lvl, threadIdx.x,
                   blockDim.x);
    side /= sb;
    lvl += (sb == 4) ? 2 : 1;
    float* t = src; src = dst; dst = t;
  }
  __syncthreads();
  return src[0];
}

// Coarse levels Lt+1..n from the (H/T) x (W/T) image of tile means in img
// (scratch: img2, same size / 16), then the scaling coefficients A_n.  WARP:
// run by one warp (tid = lane) instead of the whole block.
template <int OUT, bool WARP>
__device__ void coarse_levels_t(const ShiftArgs& a, const ShiftParam* p, int s, int c, float* img,
                                float* img2, int tid, int nthr) {
  const Geometry& g = a.g;
  int rows = g.tiles_r, cols = g.tiles_c, lvl = g.Lt;
  float* src = img;
  float* dst = img2;
  while (lvl < g.n) {
    const int sb = (g.n - lvl >= 2) ? 4 : 2;
    if (WARP) __syncwarp(); else __syncthreads();
    haar_pass<OUT>(a, p, s, c, src, dst, rows, cols, lvl, sb, 0, 0, tid, nthr);
    rows /= sb;
    cols /= sb;
    lvl += (sb == 4) ? 2 : 1;
    float* t = src; src = dst; dst = t;
  }
  if (WARP) __syncwarp(); else __syncthreads();
  for (int k = tid; k < g.q; k += nthr) {
    float v = src[k];
    if (p != nullptr && ((p->perm_mask >> (g.n + 1)) & 1u)) v = perm_value(a, *p, c, g.n + 1, 0, 0, k);
    put<OUT>(a, s, c, k, v);
  }
  if (WARP) __syncwarp(); else __syncthreads();
}

// img[k] = src[k] for k < n by threads tid, tid + nthr, ...: eight L2 loads
// in flight per thread (a loop of load -> shared store pairs waits one L2
// round trip per element: 8 of them for the 128 tile means of a 16 x 16-tile
// plane at 16 threads per plane)
__device__ __forceinline__ void gather_means(float* img, const float* src, int n, int tid, int nthr) {
  for (int k0 = tid; k0 < n; k0 += 8 * nthr) {
    float r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = (k0 + u * nthr < n) ? __ldcg(src + k0 + u * nthr) : 0.0f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (k0 + u * nthr < n) img[k0 + u * nthr] = r[u];
  }
}

template <int OUT>
__device__ __forceinline__ void coarse_levels(const ShiftArgs& a, const ShiftParam* p, int s, int c, float* img,
                                              float* img2) {
  coarse_levels_t<OUT, false>(a, p, s, c, img, img2, threadIdx.x, blockDim.x);
}

template <int OUT>
__device__ __forceinline__ void coarse_levels_warp(const ShiftArgs& a, const ShiftParam* p, int s, int c,
                                                   float* img, float* img2, int lane) {
  coarse_levels_t<OUT, true>(a, p, s, c, img, img2, lane, 32);
}

// ------------------------------------------------------------------ kernels

// One CTA per (tile, shift).  Shared memory: [window (T+1)^2 | pixels CG*T*T |
// scratch (T/4)^2 + 8] floats.
template <int KIND, int OUT>
__global__ void __launch_bounds__(kThreads) k_shift(ShiftArgs a) {
  extern __shared__ __align__(16) float smem[];
  pdl_wait();
  __shared__ int s_last;
  const Geometry& g = a.g;
  const int T = g.T;
  const int tile = blockIdx.x;
  const int s = blockIdx.y;
  const int cgrp = blockIdx.z;            // channel group of this CTA
  const int tr = tile / g.tiles_c, tc = tile - tr * g.tiles_c;
  const int CG = (KIND == KIND_ROTATE) ? kRotChannels : 1;
  const int win = (KIND == KIND_TRANSLATE) ? (T + 1) * (T + 1) : 0;
  const int winr = (win + 3) & ~3;
  float* wnd = smem;
  float* pbuf = smem + winr;
  float* sbuf = pbuf + CG * T * T;
  const ShiftParam* p = (KIND == KIND_COPY) ? nullptr : (a.prm + s);
  ShiftParam pr;
  if (p != nullptr) pr = *p;
  const int i_org = tr * T, j_org = tc * T;

  for (int c0 = cgrp * CG; c0 < g.C && c0 < (cgrp + 1) * CG; c0 += CG) {
    const int cgn = min(CG, g.C - c0);
    if (KIND == KIND_TRANSLATE) {
      const float* F = a.pix + (long long)c0 * g.N;
      const int wp = T + 1;
      __syncthreads();
      for (int e = threadIdx.x; e < wp * wp; e += blockDim.x) {
        const int wi = e / wp, wj = e - wi * wp;
        int i = i_org - pr.ky - 1 + wi, j = j_org - pr.kx - 1 + wj;
        ext_index(i, j, g.H, g.W, g.boundary);
        wnd[e] = __ldg(F + (long long)i * g.W + j);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
        const int ii = e / T, jj = e - ii * T;
        const float* w0 = wnd + ii * wp + jj;
        const float top = pr.wx0 * w0[1] + pr.wx1 * w0[0];          // row i - ky - 1
        const float bot = pr.wx0 * w0[wp + 1] + pr.wx1 * w0[wp];    // row i - ky
        pbuf[e] = pr.wy0 * bot + pr.wy1 * top;
      }
    } else if (KIND == KIND_ROTATE) {
      __syncthreads();
      const float4* rt = a.rtab + (long long)s * a.rt_stride;
      const float4* tex = reinterpret_cast<const float4*>(a.pix) + (long long)cgrp * g.N * 2;
      for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
        const int ii = e / T, jj = e - ii * T;
        const int i = i_org + ii, j = j_org + jj;
        const RotSrc o = rot_source(__ldg(a.rows + i), __ldg(rt + 2 * g.W + 2 * i), __ldg(rt + 2 * g.W + 2 * i + 1),
                                    __ldg(rt + j), rt + g.W, a.rows, pr.a_px, a.u_scale, a.v_scale, g.H, g.W);
        int t0, t1;
        rot_taps(o, g.H, g.W, g.boundary, t0, t1);
        const float4 p0 = __ldg(tex + 2 * t0), p1 = __ldg(tex + 2 * t1);
        pbuf[e] = rot_lerp(p0.x, p0.y, p1.x, p1.y, o.fu, o.fv);
        if (cgn > 1) pbuf[T * T + e] = rot_lerp(p0.z, p0.w, p1.z, p1.w, o.fu, o.fv);
        if (cgn > 2) {
          const float4 q0 = __ldg(tex + 2 * t0 + 1), q1 = __ldg(tex + 2 * t1 + 1);
          pbuf[2 * T * T + e] = rot_lerp(q0.x, q0.y, q1.x, q1.y, o.fu, o.fv);
        }
      }
    } else {  // KIND_COPY: forward transform of maps [batch][H][W]
      const float* F = a.pix + (long long)s * g.N;
      __syncthreads();
      if (T >= 4) {
        for (int e = threadIdx.x; e < T * T / 4; e += blockDim.x) {
          const int ii = (4 * e) / T, jj = 4 * e - ii * T;
          *reinterpret_cast<float4*>(pbuf + 4 * e) =
              __ldg(reinterpret_cast<const float4*>(F + (long long)(i_org + ii) * g.W + j_org + jj));
        }
      } else {
        for (int e = threadIdx.x; e < T * T; e += blockDim.x) {
          const int ii = e / T, jj = e - ii * T;
          pbuf[e] = __ldg(F + (long long)(i_org + ii) * g.W + j_org + jj);
        }
      }
    }
    for (int ci = 0; ci < cgn; ++ci) {
      const int c = c0 + ci;
      const float m = tile_levels<OUT>(a, p, s, c, pbuf + ci * T * T, sbuf, tr, tc);
      if (threadIdx.x == 0) {
        if (a.means != nullptr)
          a.means[((long long)s * g.C + c) * g.n_tiles + tile] = m;
        else  // forward transform: stash the tile mean in the coarse region of the output
          reinterpret_cast<float*>(a.out)[(long long)s * a.st_s + (long long)c * a.st_c + tile] = m;
      }
      __syncthreads();
    }
  }

  if (a.counters == nullptr) return;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.counters + s, 1u);
    s_last = (t == (unsigned)(g.n_tiles * gridDim.z - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float* img = pbuf;
  float* img2 = pbuf + ((g.n_tiles + 3) & ~3);   // float4-aligned
  for (int c = 0; c < g.C; ++c) {
    gather_means(img, a.means + ((long long)s * g.C + c) * g.n_tiles, (int)g.n_tiles, threadIdx.x, blockDim.x);
    coarse_levels<OUT>(a, p, s, c, img, img2);
  }
  if (threadIdx.x == 0) a.counters[s] = 0u;
}

// Morton (Z-order) coordinates: x from the even bits, y from the odd bits.
__device__ __forceinline__ int morton_x(int t) {
  return (t & 1) | ((t >> 1) & 2) | ((t >> 2) & 4) | ((t >> 3) & 8) | ((t >> 4) & 16);
}
__device__ __forceinline__ int morton_y(int t) { return morton_x(t >> 1); }

// One level of the transform on 4 values held by Morton-consecutive lane
// groups (lanes base + {0, st, 2 st, 3 st} = top-left, top-right,
// bottom-left, bottom-right): every lane gets the merged scaling value; the
// first three members write the H, V and D coefficient of block
// (by >> (lvl - 2), bx >> (lvl - 2)) of the tile at level lvl, where (by, bx)
// is the lane's 4 x 4 block; only lanes below `limit` write.  All 32 lanes
// must call it.
template <int OUT>
__device__ __forceinline__ float merge4(const ShiftArgs& a, const ShiftParam* p, int s, int c, float A, int lane,
                                        int st, int sh, int lvl, int i0, int j0, int by, int bx, int limit = 32) {
  const int base = lane & ~(4 * st - 1);
  const float e0 = __shfl_sync(0xffffffffu, A, base);
  const float e1 = __shfl_sync(0xffffffffu, A, base + st);
  const float e2 = __shfl_sync(0xffffffffu, A, base + 2 * st);
  const float e3 = __shfl_sync(0xffffffffu, A, base + 3 * st);
  const int m = (lane - base) >> sh;
  if ((lane & (st - 1)) == 0 && m < 3 && lane < limit) {
    const float d = (m == 0) ? 0.5f * ((e1 + e3) - (e0 + e2))
                  : (m == 1) ? 0.5f * ((e2 + e3) - (e0 + e1)) : 0.5f * ((e0 + e3) - (e1 + e2));
    const Geometry& g = a.g;
    const int gl = g.q << (2 * (g.n - lvl));
    const int r = (i0 >> lvl) + (by >> (lvl - 2)), col = (j0 >> lvl) + (bx >> (lvl - 2));
    const int k = gl * (1 + m) + r * (g.W >> lvl) + col;
    if (k < a.K) {
      float v = d;
      if (p != nullptr && ((p->perm_mask >> lvl) & 1u)) v = perm_value(a, *p, c, lvl, m, r, col);
      store_at<OUT>(a, (long long)s * a.st_s + (long long)c * a.st_c + (long long)k * a.st_k, v);
    }
  }
  return 0.5f * ((e0 + e1) + (e2 + e3));
}

__device__ __forceinline__ float f4c(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Bilinear resample of a translated 4 x 4 block from the source window held
// as 5 rows x 8 aligned columns: row r, column q of the block reads window
// columns O + q and O + q + 1 (O = the shift's column phase, uniform per
// launch); wx1 weights column q, wx0 column q + 1 (likewise along rows).
template <int O>
__device__ __forceinline__ void bilin_tr(const float4 (&v)[5][2], float wx0, float wx1, float wy0, float wy1,
                                         float (&x)[16]) {
  float h[5][4];
#pragma unroll
  for (int r = 0; r < 5; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c0 = O + q, c1 = O + q + 1;
      const float w0 = f4c(v[r][c0 >> 2], c0 & 3), w1 = f4c(v[r][c1 >> 2], c1 & 3);
      h[r][q] = wx0 * w1 + wx1 * w0;
    }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) x[4 * r + q] = wy0 * h[r + 1][q] + wy1 * h[r][q];
}

// Levels 1-2 of the thread's 4 x 4 block: writes the 15 detail coefficients
// and returns the level-2 scaling value.  fast: float32 output, k
// contiguous, no permuted level, levels 1-2 untruncated, and x pre-scaled by
// 1/2 (exact), so that level 1 needs no multiplies; the level-1
// coefficients then leave as three 2 x 2 patches of float2 stores.
template <int OUT>
__device__ __forceinline__ float levels12(const ShiftArgs& a, const ShiftParam* p, int s, int c, const float (&x)[16],
                                          bool fast, int tr, int tc, int by, int bx) {
  const Geometry& g = a.g;
  const int T = g.T;
  if (!fast) return block4<OUT>(a, p, s, c, x, 0, tr * T, tc * T, by, bx);
  const int g1 = g.q << (2 * (g.n - 1)), g2 = g.q << (2 * (g.n - 2));
  float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)c * a.st_c;
  float A1[4], D1[3][4];
#pragma unroll
  for (int sa = 0; sa < 2; ++sa)
#pragma unroll
    for (int sc = 0; sc < 2; ++sc) {
      const float ea = x[(2 * sa) * 4 + 2 * sc], eb = x[(2 * sa) * 4 + 2 * sc + 1];
      const float ec = x[(2 * sa + 1) * 4 + 2 * sc], ed = x[(2 * sa + 1) * 4 + 2 * sc + 1];
      A1[2 * sa + sc] = (ea + eb) + (ec + ed);
      D1[0][2 * sa + sc] = (eb + ed) - (ea + ec);
      D1[1][2 * sa + sc] = (ec + ed) - (ea + eb);
      D1[2][2 * sa + sc] = (ea + ed) - (eb + ec);
    }
  const int cols1 = g.W >> 1, cols2 = g.W >> 2;
  const int r1 = ((tr * T) >> 1) + 2 * by, c1 = ((tc * T) >> 1) + 2 * bx;
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float* pb = ob + g1 * (1 + b) + r1 * cols1 + c1;
    *reinterpret_cast<float2*>(pb) = make_float2(D1[b][0], D1[b][1]);
    *reinterpret_cast<float2*>(pb + cols1) = make_float2(D1[b][2], D1[b][3]);
  }
  const float ea = A1[0], eb = A1[1], ec = A1[2], ed = A1[3];
  if (4 * g2 <= a.K) {
    float* p2 = ob + (((tr * T) >> 2) + by) * cols2 + ((tc * T) >> 2) + bx;
    p2[g2] = 0.5f * ((eb + ed) - (ea + ec));
    p2[2 * g2] = 0.5f * ((ec + ed) - (ea + eb));
    p2[3 * g2] = 0.5f * ((ea + ed) - (eb + ec));
  }
  return 0.5f * ((ea + eb) + (ec + ed));
}

__device__ __forceinline__ void named_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// merge4 for the fast path (float32, k contiguous, no permuted level): the
// stores go to the (shift, channel) plane `ob` directly.
__device__ __forceinline__ float merge4f(float* ob, const Geometry& g, int K, float A, int lane, int st, int sh,
                                         int lvl, int i0, int j0, int by, int bx, int limit = 32) {
  const int base = lane & ~(4 * st - 1);
  const float e0 = __shfl_sync(0xffffffffu, A, base);
  const float e1 = __shfl_sync(0xffffffffu, A, base + st);
  const float e2 = __shfl_sync(0xffffffffu, A, base + 2 * st);
  const float e3 = __shfl_sync(0xffffffffu, A, base + 3 * st);
  const int m = (lane - base) >> sh;
  if ((lane & (st - 1)) == 0 && m < 3 && lane < limit) {
    const float d = (m == 0) ? 0.5f * ((e1 + e3) - (e0 + e2))
                  : (m == 1) ? 0.5f * ((e2 + e3) - (e0 + e1)) : 0.5f * ((e0 + e3) - (e1 + e2));
    const int gl = g.q << (2 * (g.n - lvl));
    const int k = gl * (1 + m) + ((i0 >> lvl) + (by >> (lvl - 2))) * (g.W >> lvl) + (j0 >> lvl) + (bx >> (lvl - 2));
    if (k < K) ob[k] = d;
  }
  return 0.5f * ((e0 + e1) + (e2 + e3));
}

// Register path for 32 x 32 and 64 x 64 tiles: every thread resamples its own
// 4 x 4 block of output pixels for up to CG channels straight from
// the L2-resident pixel map (translation: a 5 x 8 aligned window of float4
// loads per channel; rotation: 4 bilinear taps per pixel and channel at
// shared coordinates), runs levels 1-2 in registers and writes them; levels
// 3-4 merge Morton-consecutive lanes by shuffles.  The other warps then
// leave, and warp 0 finishes the tile's levels 5-6 from shared memory, hands
// the tile mean on, and (last tile of a shift) runs the coarse levels.
// blockDim = (T/4)^2.
// SMT (rotations): the rotation's anchor-column table and the map's row table
// are first copied to shared memory, so that the two dependent table lookups
// of every pixel are shared-memory loads.
template <int KIND, int OUT, int CG, bool SMT = false>
__global__ void __launch_bounds__(kThreads, KIND == KIND_ROTATE ? 3 : 4) k_shift_reg(ShiftArgs a) {
  extern __shared__ __align__(16) float smem[];
  const Geometry& g = a.g;
  const int T = g.T;
  const int nb = T >> 2;
  const int tile = blockIdx.x, s = blockIdx.y, cgrp = blockIdx.z;
  const int tr = tile / g.tiles_c, tc = tile - tr * g.tiles_c;
  const int c0 = cgrp * CG;
  const int cgn = min(CG, g.C - c0);
  __shared__ ShiftParam s_prm;
  pdl_wait();
  if (KIND != KIND_COPY && threadIdx.x == 0) s_prm = a.prm[s];
  __syncthreads();
  const ShiftParam* p = (KIND == KIND_COPY) ? nullptr : &s_prm;
  // Morton (Z-order) placement of the thread's 4 x 4 block: the 4, 16, 64 ...
  // blocks that merge at levels 3, 4, 5 ... are consecutive threads
  const int by = morton_y(threadIdx.x), bx = morton_x(threadIdx.x);
  const int i0 = tr * T + 4 * by, j0 = tc * T + 4 * bx;
  const int Wm = g.W - 1;
  const int g1 = g.q << (2 * (g.n - 1));
  // the fast path stores 8-byte vectors: the output must be 8-byte aligned
  const bool fast = OUT == HAAR_OUT_F32 && a.st_k == 1 && a.scale == 1.0f && (p == nullptr || p->perm_mask == 0u) &&
                    4 * g1 <= a.K && g.n >= 2 && (reinterpret_cast<uintptr_t>(a.out) & 7) == 0;
  const float hsc = fast ? 0.5f : 1.0f;

  float a2[CG];
  if (KIND == KIND_TRANSLATE) {
    const ShiftParam pr = *p;
    // source rows (pole crossings mirror the row and move half a turn) and
    // the 16-byte aligned first column of each row's window
    const int o = (-(pr.kx + 1)) & 3;                 // column phase, the same for every row
    int ro[5], ca[5];
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      int i = i0 - pr.ky - 1 + r, sh = 0;
      if (g.boundary == HAAR_BOUNDARY_TORUS) {
        i &= (g.H - 1);
      } else {
#pragma unroll 1
        for (int it = 0; it < 8 && (i < 0 || i >= g.H); ++it) {
          i = (i < 0) ? -1 - i : 2 * g.H - 1 - i;
          sh ^= 1;
        }
      }
      ro[r] = i * g.W;
      ca[r] = j0 - pr.kx - 1 + (sh ? (g.W >> 1) : 0) - o;
    }
    const float wx0 = pr.wx0, wx1 = pr.wx1, wy0 = pr.wy0 * hsc, wy1 = pr.wy1 * hsc;
#pragma unroll
    for (int ci = 0; ci < CG; ++ci) {
      if (ci < cgn) {
        const float* F = a.pix + (long long)(c0 + ci) * g.N;
        float4 v[5][2];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
          v[r][0] = __ldg(reinterpret_cast<const float4*>(F + ro[r] + (ca[r] & Wm)));
          v[r][1] = __ldg(reinterpret_cast<const float4*>(F + ro[r] + ((ca[r] + 4) & Wm)));
        }
        float x[16];
        switch (o) {
          case 0: bilin_tr<0>(v, wx0, wx1, wy0, wy1, x); break;
          case 1: bilin_tr<1>(v, wx0, wx1, wy0, wy1, x); break;
          case 2: bilin_tr<2>(v, wx0, wx1, wy0, wy1, x); break;
          default: bilin_tr<3>(v, wx0, wx1, wy0, wy1, x); break;
        }
        a2[ci] = levels12<OUT>(a, p, s, c0 + ci, x, fast, tr, tc, by, bx);
      }
    }
  } else if (KIND == KIND_ROTATE) {
    // row pairs: the two rows' 8 pixels per channel finish their two level-1
    // blocks at once, so only one row pair of pixels is live at a time
    const ShiftParam pr = *p;
    const float4* rt = a.rtab + (long long)s * a.rt_stride;
    const float4* tex = reinterpret_cast<const float4*>(a.pix) + (long long)cgrp * g.N * 2;
    const float4* colal = rt + g.W;
    const float4* rowtab = a.rows;
    if constexpr (SMT) {
      float4* st = reinterpret_cast<float4*>(smem + a.tab_off);
      for (int e = threadIdx.x; e < g.W + g.H; e += blockDim.x)
        st[e] = (e < g.W) ? __ldg(rt + g.W + e) : __ldg(a.rows + (e - g.W));
      __syncthreads();
      colal = st;
      rowtab = st + g.W;
    }
    float4 ps[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ps[q] = __ldg(rt + j0 + q);
    // the row loops stay rolled: a row's body (4 pixels' coordinates) is
    // large, and unrolled copies of it measured slower (instruction fetch stalls)
    float A1[CG][4];
#pragma unroll 1
    for (int rp = 0; rp < 2; ++rp) {
      float x[CG][8];
#pragma unroll 1
      for (int rr = 0; rr < 2; ++rr) {
        const int i = i0 + 2 * rp + rr;
        const float4 th = __ldg(a.rows + i), ab = __ldg(rt + 2 * g.W + 2 * i), cd = __ldg(rt + 2 * g.W + 2 * i + 1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const RotSrc o = rot_source<!SMT>(th, ab, cd, ps[q], colal, rowtab, pr.a_px, a.u_scale, a.v_scale, g.H, g.W);
          int t0, t1;
          rot_taps(o, g.H, g.W, g.boundary, t0, t1);
          float e0[8], e1[8];
          ld_texel(tex + 2 * t0, e0);
          ld_texel(tex + 2 * t1, e1);
          const float w = hsc;
#pragma unroll
          for (int ci = 0; ci < CG; ++ci)
            if (ci < cgn) {
              const float val = w * rot_lerp(e0[2 * ci], e0[2 * ci + 1], e1[2 * ci], e1[2 * ci + 1], o.fu, o.fv);
              if (rr == 0) x[ci][q] = val; else x[ci][4 + q] = val;
            }
        }
      }
      // level 1 of the row pair's two 2 x 2 blocks (pixels pre-scaled by 1/2 on the fast path)
#pragma unroll
      for (int ci = 0; ci < CG; ++ci) {
        if (ci < cgn) {
          float D[3][2];
#pragma unroll
          for (int sc = 0; sc < 2; ++sc) {
            const float ea = x[ci][2 * sc], eb = x[ci][2 * sc + 1];
            const float ec = x[ci][4 + 2 * sc], ed = x[ci][4 + 2 * sc + 1];
            const float h = fast ? 1.0f : 0.5f;
            const float av = h * ((ea + eb) + (ec + ed));
            if (rp == 0) A1[ci][sc] = av; else A1[ci][2 + sc] = av;
            D[0][sc] = h * ((eb + ed) - (ea + ec));
            D[1][sc] = h * ((ec + ed) - (ea + eb));
            D[2][sc] = h * ((ea + ed) - (eb + ec));
          }
          const int r1 = ((tr * T) >> 1) + 2 * by + rp, c1 = ((tc * T) >> 1) + 2 * bx;
          if (fast) {
            float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)(c0 + ci) * a.st_c;
            const int cols1 = g.W >> 1;
#pragma unroll
            for (int b = 0; b < 3; ++b)
              *reinterpret_cast<float2*>(ob + g1 * (1 + b) + r1 * cols1 + c1) = make_float2(D[b][0], D[b][1]);
          } else {
#pragma unroll
            for (int sc = 0; sc < 2; ++sc) emit<OUT>(a, p, s, c0 + ci, 1, r1, c1 + sc, D[0][sc], D[1][sc], D[2][sc]);
          }
        }
      }
    }
    // level 2 of the thread's block
#pragma unroll
    for (int ci = 0; ci < CG; ++ci) {
      if (ci < cgn) {
        const float ea = A1[ci][0], eb = A1[ci][1], ec = A1[ci][2], ed = A1[ci][3];
        emit<OUT>(a, p, s, c0 + ci, 2, ((tr * T) >> 2) + by, ((tc * T) >> 2) + bx, 0.5f * ((eb + ed) - (ea + ec)),
                  0.5f * ((ec + ed) - (ea + eb)), 0.5f * ((ea + ed) - (eb + ec)));
        a2[ci] = 0.5f * ((ea + eb) + (ec + ed));
      }
    }
  } else {  // KIND_COPY
    const float* F = a.pix + (long long)s * g.N;
    float x[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(F + (long long)(i0 + r) * g.W + j0));
      x[4 * r] = t.x * hsc; x[4 * r + 1] = t.y * hsc; x[4 * r + 2] = t.z * hsc; x[4 * r + 3] = t.w * hsc;
    }
    a2[0] = levels12<OUT>(a, p, s, 0, x, fast, tr, tc, by, bx);
  }

  // levels 3 and 4: merges of 4 Morton-consecutive lanes (strides 1 and 4);
  // one value per 16 lanes remains and goes to shared memory
  const int lane = threadIdx.x & 31;
  const int nthreads = nb * nb;
  const int nwarps = nthreads >> 5;
  const int groups = nthreads >> 4;
  float* sA = smem;                                 // [CG][groups]
#pragma unroll
  for (int ci = 0; ci < CG; ++ci) {
    if (ci < cgn) {
      float A;
      if (fast) {
        float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)(c0 + ci) * a.st_c;
        A = merge4f(ob, g, a.K, a2[ci], lane, 1, 0, 3, tr * T, tc * T, by, bx);
        A = merge4f(ob, g, a.K, A, lane, 4, 2, 4, tr * T, tc * T, by, bx);
      } else {
        A = merge4<OUT>(a, p, s, c0 + ci, a2[ci], lane, 1, 0, 3, tr * T, tc * T, by, bx);
        A = merge4<OUT>(a, p, s, c0 + ci, A, lane, 4, 2, 4, tr * T, tc * T, by, bx);
      }
      if ((lane & 15) == 0) sA[ci * groups + (threadIdx.x >> 4)] = A;
    }
  }
  // warps that finish a channel's tile below stay; the others leave
  const int wid = threadIdx.x >> 5;
  if (wid >= cgn) {
    named_arrive(1, nthreads);
    return;
  }
  named_sync(1, nthreads);
  pdl_trigger();                                  // the tile's levels 1-4 are written

  // warp w: levels 5..Lt of channels w, w + nwarps, ... on the `groups`
  // values (a Morton-ordered grid of 16 x 16-pixel blocks), then the tile
  // mean; the last arrival of a shift runs its coarse levels
  const int gy = morton_y(lane) << 2, gx = morton_x(lane) << 2;
  unsigned last = 0;
  for (int ci = wid; ci < cgn; ci += nwarps) {
    const int c = c0 + ci;
    float B = (lane < groups) ? sA[ci * groups + lane] : 0.0f;
    int st2 = 1, sh2 = 0;
    float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)c * a.st_c;
    for (int lvl = 4; lvl < g.Lt; ++lvl) {
      B = fast ? merge4f(ob, g, a.K, B, lane, st2, sh2, lvl + 1, tr * T, tc * T, gy, gx, groups)
               : merge4<OUT>(a, p, s, c, B, lane, st2, sh2, lvl + 1, tr * T, tc * T, gy, gx, groups);
      st2 *= 4;
      sh2 += 2;
    }
    if (lane == 0) {
      if (a.means != nullptr)
        a.means[((long long)s * g.C + c) * g.n_tiles + tile] = B;
      else
        reinterpret_cast<float*>(a.out)[(long long)s * a.st_s + (long long)c * a.st_c + tile] = B;
    }
    if (a.counters != nullptr && lane == 0) {
      __threadfence();
      const unsigned t = atomicAdd(a.counters + s, 1u);
      if (t == (unsigned)(g.n_tiles * g.C - 1)) last = 1u;
    }
  }
  if (a.counters == nullptr) return;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  // past sA, which the CTA's other warps may still be reading
  float* img = smem + ((CG * groups + 3) & ~3);
  float* img2 = img + ((g.n_tiles + 3) & ~3);   // float4-aligned
  for (int c = 0; c < g.C; ++c) {
    gather_means(img, a.means + ((long long)s * g.C + c) * g.n_tiles, (int)g.n_tiles, lane, 32);
    coarse_levels_warp<OUT>(a, p, s, c, img, img2, lane);
  }
  if (lane == 0) a.counters[s] = 0u;
}

// ------------------------------------------------------------------ translation, 8 x 8 blocks
// F32 translations into a k-contiguous layout (batches of many shifts):
// CTA = one 64 x 64 output tile of one shift, all channels, thread per 8 x 8
// block of output pixels (64 threads).  Per channel a thread streams the 9
// source rows of its block's window (3 aligned float4 loads per row) from
// the tile's window staged in shared memory by one TMA box of the plan's
// extended map, or, without that map, from the pixel map with the rows'
// offsets (pole mirroring, column wrap) computed once per thread; it lerps
// each row horizontally and
// each pair of rows vertically (weights pre-scaled by 1/2, exact), and
// finishes levels 1-3 of its block in registers: level-1 details leave as
// one float4 per row and band, level 2 as float2, level 3 as scalars.  The
// level-3 means of the tile go through shared memory to levels 4-6, and the
// last CTA of a shift runs the coarse levels.  Against the 4 x 4 block of
// k_shift_reg, a thread's window loads, row addresses and stores are shared
// by 4x the outputs, and no level needs a shuffle merge.
constexpr int kTr8Threads = 64;

template <int O>
__device__ __forceinline__ void tr8_hlerp(const float4 (&v)[3], float wx0, float wx1, float (&h)[8]) {
  const float w[12] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y,
                       v[1].z, v[1].w, v[2].x, v[2].y, v[2].z, v[2].w};
#pragma unroll
  for (int q = 0; q < 8; ++q) h[q] = wx0 * w[O + q + 1] + wx1 * w[O + q];
}

// the 3 float4 of window row `off` (row * W + first aligned column); wrap:
// the window crosses the last column, each float4 column wraps separately
template <bool SM = false>
__device__ __forceinline__ void tr8_load(const float* __restrict__ F, int off, bool wrap, int Wm,
                                         float4 (&v)[3]) {
  if (SM) {                                       // the window staged in shared memory
    const float4* p = reinterpret_cast<const float4*>(F + off);
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
  } else if (!wrap) {
    const float4* p = reinterpret_cast<const float4*>(F + off);
    v[0] = __ldg(p);
    v[1] = __ldg(p + 1);
    v[2] = __ldg(p + 2);
  } else {
    const int c = off & Wm, rb = off - c;
#pragma unroll
    for (int m = 0; m < 3; ++m) v[m] = __ldg(reinterpret_cast<const float4*>(F + rb + ((c + 4 * m) & Wm)));
  }
}

// Signed-permutation levels (dyadic integer shifts): the `cnt` coefficients
// of row r, columns c0.. of level lvl, every band, taken from the input
// (kept out of line: the hot path only tests the level's bit).
__device__ __noinline__ void tr8_perm_row(const ShiftArgs& a, const ShiftParam& pr, int c, int lvl, int r, int c0,
                                          int cnt, float* __restrict__ ob) {
  const Geometry& g = a.g;
  const long long gl = (long long)g.q << (2 * (g.n - lvl));
  float* p = ob + (long long)r * (g.W >> lvl) + c0;
  for (int b = 0; b < cnt; ++b)
    for (int m = 0; m < 3; ++m) p[(1 + m) * gl + b] = perm_value(a, pr, c, lvl, m, r, c0 + b);
}

// Rows 4u .. 4u + 3 of a channel's 8 x 8 block (source rows 4u + 1 .. 4u + 4
// at offsets o1..o4; hA holds the horizontally lerped row 4u and leaves with
// row 4u + 4): level 1 of its two row pairs and level 2 of its two 2 x 2
// blocks; a2 receives the two level-2 means.
template <int O, bool SM>
__device__ __forceinline__ void tr8_half(const ShiftArgs& a, const ShiftParam& pr, int c, const float* __restrict__ F,
                                         float* __restrict__ ob, int o1, int o2, int o3, int o4, bool wrap, int u,
                                         int i0, int j0, float (&hA)[8], float (&a2)[2]) {
  const Geometry& g = a.g;
  const int Wm = g.W - 1;
  const float wx0 = pr.wx0, wx1 = pr.wx1, wy0 = 0.5f * pr.wy0, wy1 = 0.5f * pr.wy1;
  const long long g1 = (long long)g.q << (2 * (g.n - 1)), g2 = g1 >> 2;
  const int cols1 = g.W >> 1, cols2 = g.W >> 2;
  const uint32_t pm = pr.perm_mask;
  float4 v[3];
  float hB[8], hC[8];
  float A1[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    tr8_load<SM>(F, h ? o3 : o1, wrap, Wm, v);
    tr8_hlerp<O>(v, wx0, wx1, hB);
    tr8_load<SM>(F, h ? o4 : o2, wrap, Wm, v);
    tr8_hlerp<O>(v, wx0, wx1, hC);
    float Dh[4], Dv[4], Dd[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float ea = wy0 * hB[2 * b] + wy1 * hA[2 * b], eb = wy0 * hB[2 * b + 1] + wy1 * hA[2 * b + 1];
      const float ec = wy0 * hC[2 * b] + wy1 * hB[2 * b], ed = wy0 * hC[2 * b + 1] + wy1 * hB[2 * b + 1];
      A1[h][b] = (ea + eb) + (ec + ed);
      Dh[b] = (eb + ed) - (ea + ec);
      Dv[b] = (ec + ed) - (ea + eb);
      Dd[b] = (ea + ed) - (eb + ec);
    }
    const int r1 = (i0 >> 1) + 2 * u + h, c1 = j0 >> 1;
    float* p1 = ob + (long long)r1 * cols1 + c1;
    *reinterpret_cast<float4*>(p1 + g1) = make_float4(Dh[0], Dh[1], Dh[2], Dh[3]);
    *reinterpret_cast<float4*>(p1 + 2 * g1) = make_float4(Dv[0], Dv[1], Dv[2], Dv[3]);
    *reinterpret_cast<float4*>(p1 + 3 * g1) = make_float4(Dd[0], Dd[1], Dd[2], Dd[3]);
    if (pm & 2u) tr8_perm_row(a, pr, c, 1, r1, c1, 4, ob);
#pragma unroll
    for (int q = 0; q < 8; ++q) hA[q] = hC[q];
  }
  float Dh[2], Dv[2], Dd[2];
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    const float ea = A1[0][2 * w], eb = A1[0][2 * w + 1], ec = A1[1][2 * w], ed = A1[1][2 * w + 1];
    a2[w] = 0.5f * ((ea + eb) + (ec + ed));
    Dh[w] = 0.5f * ((eb + ed) - (ea + ec));
    Dv[w] = 0.5f * ((ec + ed) - (ea + eb));
    Dd[w] = 0.5f * ((ea + ed) - (eb + ec));
  }
  const int r2 = (i0 >> 2) + u, c2 = j0 >> 2;
  float* p2 = ob + (long long)r2 * cols2 + c2;
  *reinterpret_cast<float2*>(p2 + g2) = make_float2(Dh[0], Dh[1]);
  *reinterpret_cast<float2*>(p2 + 2 * g2) = make_float2(Dv[0], Dv[1]);
  *reinterpret_cast<float2*>(p2 + 3 * g2) = make_float2(Dd[0], Dd[1]);
  if (pm & 4u) tr8_perm_row(a, pr, c, 2, r2, c2, 2, ob);
}

// Levels 1-3 of one channel's 8 x 8 block; returns the level-3 mean.
// ob = the (shift, channel) plane, (i0, j0) the block's first pixel.  The
// two halves run as a rolled loop: the unrolled block (x 4 column phases)
// measured slower, bound by instruction fetch.
template <int O, bool SM = false>
__device__ __forceinline__ float tr8_block(const ShiftArgs& a, const ShiftParam& pr, int c, const float* __restrict__ F,
                                           float* __restrict__ ob, const int (&off)[9], bool wrap, int i0, int j0) {
  const Geometry& g = a.g;
  float4 v[3];
  float hA[8];
  tr8_load<SM>(F, off[0], wrap, g.W - 1, v);
  tr8_hlerp<O>(v, pr.wx0, pr.wx1, hA);
  float a20[2], a21[2];
#pragma unroll 1
  for (int u = 0; u < 2; ++u) {
    float t[2];
    tr8_half<O, SM>(a, pr, c, F, ob, u ? off[5] : off[1], u ? off[6] : off[2], u ? off[7] : off[3],
                u ? off[8] : off[4], wrap, u, i0, j0, hA, t);
    if (u == 0) { a20[0] = t[0]; a20[1] = t[1]; } else { a21[0] = t[0]; a21[1] = t[1]; }
  }
  // level 3
  const float ea = a20[0], eb = a20[1], ec = a21[0], ed = a21[1];
  const long long g3 = (long long)g.q << (2 * (g.n - 3));
  const int r3 = i0 >> 3, c3 = j0 >> 3;
  float* p3 = ob + (long long)r3 * (g.W >> 3) + c3;
  p3[g3] = 0.5f * ((eb + ed) - (ea + ec));
  p3[2 * g3] = 0.5f * ((ec + ed) - (ea + eb));
  p3[3 * g3] = 0.5f * ((ea + ed) - (eb + ec));
  if (pr.perm_mask & 8u) tr8_perm_row(a, pr, c, 3, r3, c3, 1, ob);
  return 0.5f * ((ea + eb) + (ec + ed));
}

// One level (4 <= lvl <= 6) of the tile from the previous level's means in
// shared memory: work item e = (channel, block row u, block column v) of an
// nb x nb grid of 2 x 2 blocks (the source grid is 2 nb wide).
__device__ __forceinline__ void tr8_level(const ShiftArgs& a, const ShiftParam& pr, int s, int lvl, int nb,
                                          const float* src, float* dst, int tr, int tc) {
  const Geometry& g = a.g;
  const long long gl = (long long)g.q << (2 * (g.n - lvl));
  const int cols = g.W >> lvl;
  for (int e = threadIdx.x; e < g.C * nb * nb; e += blockDim.x) {
    const int c = e / (nb * nb), rem = e - c * nb * nb, u = rem / nb, w = rem - u * nb;
    const float* q = src + c * 4 * nb * nb;
    const float ea = q[(2 * u) * 2 * nb + 2 * w], eb = q[(2 * u) * 2 * nb + 2 * w + 1];
    const float ec = q[(2 * u + 1) * 2 * nb + 2 * w], ed = q[(2 * u + 1) * 2 * nb + 2 * w + 1];
    float d[3] = {0.5f * ((eb + ed) - (ea + ec)), 0.5f * ((ec + ed) - (ea + eb)), 0.5f * ((ea + ed) - (eb + ec))};
    const int r = ((tr * g.T) >> lvl) + u, col = ((tc * g.T) >> lvl) + w;
    float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)c * a.st_c;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      float x = d[m];
      if ((pr.perm_mask >> lvl) & 1u) x = perm_value(a, pr, c, lvl, m, r, col);
      ob[gl * (1 + m) + (long long)r * cols + col] = x;
    }
    dst[c * nb * nb + u * nb + w] = 0.5f * ((ea + eb) + (ec + ed));
  }
}

// Shared memory (floats): level-3 means [C][64], then the tail
// (tr8_tail_floats): level-4 [C][16], level-5 [C][4], level-6 [C] and (last
// CTA of a shift) the tile-mean image and its scratch.
template <int O>
__device__ __forceinline__ void tr8_channels(const ShiftArgs& a, const ShiftParam& pr, int s, const int (&off)[9],
                                             bool wrap, int i0, int j0, float* sA3) {
  const Geometry& g = a.g;
#pragma unroll 1
  for (int c = 0; c < g.C; ++c) {
    const float* F = a.pix + (long long)c * g.N;
    float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)c * a.st_c;
    sA3[c * 64 + threadIdx.x] = tr8_block<O>(a, pr, c, F, ob, off, wrap, i0, j0);
  }
}

// The TMA-fed form: the tile's source window of every channel (65 rows x 68
// columns of the extended map) arrives in shared memory by TMA as eight bands
// of 8 rows and the last row, each box 72 columns wide; the odd bands start 4
// columns earlier in the map, so their rows sit 4 floats (4 banks) further on
// in shared memory.  With one 65 x 68 box every block row of a warp (rows 8
// apart) started on the same banks; the bands spread a warp's 16-byte reads
// over twice as many bank groups: 7.77 M -> 5.83 M shared-load wavefronts for
// 512 shifts of RGB 128x256, and 0.418 -> 0.405 ms for 4096.  (Those reads
// are served 8 lanes at a time, and within 8 lanes, one block row, columns
// 32 floats apart still share banks; a thread-to-block assignment that gave
// each 8 lanes two block rows measured slower: 0.408 ms at 96 registers,
// 0.454 ms with spills at 72.)
constexpr int kTr8WinRows = 65, kTr8WinCols = 68;       // the window a tile reads
constexpr int kTr8BoxCols = 72, kTr8BandRows = 8, kTr8Bands = 8;
constexpr int kTr8BandFloats = kTr8BandRows * kTr8BoxCols;          // 576 floats = 18 x 128 bytes
constexpr int kTr8WinFloats = kTr8Bands * kTr8BandFloats + 96;      // + the last row, a 128-byte multiple
constexpr unsigned kTr8WinBytes = (kTr8Bands * kTr8BandRows + 1) * kTr8BoxCols * 4;
static_assert(kTr8Bands * kTr8BandRows + 1 == kTr8WinRows && kTr8BoxCols >= kTr8WinCols + 4, "window boxes");
// one window per CTA (the next channel's copy issued once the current one is
// read): 18.8 KB of shared memory; two windows in flight (6 CTAs per SM)
// measured slower (0.498 against 0.418 ms for 4096 shifts of RGB 128x256
// with the single-box window), as did the direct loads (0.439 ms)
constexpr int kTr8Windows = 1;

// Shared floats of the kernel's tail, which runs after the last window is
// consumed: the level means [C][16], [C][4] and [C] (rounded up to 4) and,
// in the last CTA of a shift, the tile-mean image and its next level.  The
// TMA-fed form puts the tail in the window's shared memory when it fits.
static long long tr8_tail_floats(int C, long long n_tiles) {
  return 20LL * C + ((C + 3) & ~3) + ((n_tiles + 3) & ~3LL) + ((n_tiles / 4 + 4) & ~3LL);
}

static bool tr8_tail_in_window(bool tma, int C, long long n_tiles) {
  return tma && tr8_tail_floats(C, n_tiles) <= (long long)kTr8Windows * kTr8WinFloats;
}

// offset in the staged window of window row R (0..64), block column bx
__device__ __forceinline__ int tr8_win_off(int R, int bx) {
  const int b = R >> 3;
  return b * kTr8BandFloats + (R & 7) * kTr8BoxCols + 4 * (b & 1) + 8 * bx;
}

// issue the window of channel c (map columns from xw, rows from yw) into w:
// the bands by mapB (72 x 8 boxes; odd bands from column xw - 4, which for
// xw = 0 reads the zero fill left of the map, columns no thread uses), the
// last row by mapR (a 72 x 1 box); all of it completes on barrier `bar`
__device__ __forceinline__ void tr8_issue(float* w, const CUtensorMap* mapB, const CUtensorMap* mapR, int xw,
                                          int yw, int c, uint32_t bar) {
  tc::mbar_arrive_tx(bar, kTr8WinBytes);
#pragma unroll
  for (int b = 0; b < kTr8Bands; ++b)
    tc::tma_load_3d(tc::smem_u32(w + b * kTr8BandFloats), mapB, xw - 4 * (b & 1), yw + kTr8BandRows * b, c, bar);
  tc::tma_load_3d(tc::smem_u32(w + kTr8Bands * kTr8BandFloats), mapR, xw, yw + kTr8Bands * kTr8BandRows, c, bar);
}
constexpr unsigned long long kTr8WaitNs = 2000000000ull;

// bounded wait on a window's barrier; false (status set) on expiry
__device__ __forceinline__ bool tr8_wait(uint32_t bar, uint32_t parity, int* status) {
  if (tc::mbar_try(bar, parity)) return true;
  const unsigned long long t0 = tc::gtimer();
  while (!tc::mbar_try(bar, parity))
    if (tc::gtimer() - t0 > kTr8WaitNs) {
      if (status != nullptr) atomicOr(status, 1 << HAAR_ERR_TIMEOUT);
      return false;
    }
  return true;
}

template <int O, int NB>
__device__ __forceinline__ void tr8_channels_tma(const ShiftArgs& a, const ShiftParam& pr, int s, const int (&off)[9],
                                                 int i0, int j0, float* sA3, float* win, uint64_t* wbar,
                                                 int* wissued, int* wdone, const CUtensorMap* mapP,
                                                 const CUtensorMap* mapR, int xw, int yw, int* s_fail) {
  const Geometry& g = a.g;
#pragma unroll 1
  for (int c = 0; c < g.C; ++c) {
    const int b = c % NB;
    float* w = win + b * kTr8WinFloats;
    if (*s_fail == 0 && !tr8_wait(tc::smem_u32(&wbar[b]), (uint32_t)(wdone[b] & 1), a.status)) *s_fail = 1;
    __syncthreads();
    const bool ok = *s_fail == 0;
    if (threadIdx.x == 0 && ok) ++wdone[b];
    float* ob = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s + (long long)c * a.st_c;
    if (ok) sA3[c * 64 + threadIdx.x] = tr8_block<O, true>(a, pr, c, w, ob, off, false, i0, j0);
    __syncthreads();                                // every thread is done with this window
    if (threadIdx.x == 0 && ok && c + NB < g.C) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tr8_issue(w, mapP, mapR, xw, yw, c + NB, tc::smem_u32(&wbar[b]));
      ++wissued[b];
    }
  }
}

// 72 registers (room for 14 CTAs per SM; shared memory allows 11: the window,
// the level-3 means and the tail in the window); 64 or 80 measured slower
template <bool TMA, int NB>
__global__ void __launch_bounds__(kTr8Threads, 14) k_shift_tr8(ShiftArgs a, const __grid_constant__ CUtensorMap mapP,
                                                                      const __grid_constant__ CUtensorMap mapR) {
  extern __shared__ __align__(16) float smem[];
  __shared__ ShiftParam s_prm;
  __shared__ int s_last;
  const Geometry& g = a.g;
  const int tile = blockIdx.x;
  const int tr = tile / g.tiles_c, tc = tile - tr * g.tiles_c;
  pdl_wait();
  const int s = a.prm[blockIdx.y].order;              // CTA rows run the shifts grouped by column phase
  if (threadIdx.x == 0) s_prm = a.prm[s];
  __syncthreads();
  const ShiftParam& pr = s_prm;          // shared: perm_value and the coarse pass take it by reference
  // the thread's block: row-major 8 x 8 grid of blocks in the tile
  const int by = threadIdx.x >> 3, bx = threadIdx.x & 7;
  const int i0 = tr * g.T + 8 * by, j0 = tc * g.T + 8 * bx;
  const int Wm = g.W - 1;
  const int o = (-(pr.kx + 1)) & 3;                       // column phase, the same for every row
  const int cb = j0 - pr.kx - 1 - o;                      // 16-byte aligned first column
  int off[9];
  bool wrap = false;
#pragma unroll
  for (int r = 0; r < 9 && !TMA; ++r) {
    int i = i0 - pr.ky - 1 + r, sh = 0;
    if (g.boundary == HAAR_BOUNDARY_TORUS) {
      i &= (g.H - 1);
    } else {
#pragma unroll 1
      for (int it = 0; it < 8 && (i < 0 || i >= g.H); ++it) {
        i = (i < 0) ? -1 - i : 2 * g.H - 1 - i;
        sh ^= 1;
      }
    }
    const int c = (cb + (sh ? (g.W >> 1) : 0)) & Wm;
    off[r] = i * g.W + c;
    wrap |= c + 12 > g.W;
  }
  // TMA: two windows at a 128-byte aligned start (the launch adds 128 bytes)
  float* win = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem) + 127) & ~uintptr_t(127));
  float* sA3 = TMA ? win + NB * kTr8WinFloats : smem;
  float* sA4 = TMA ? win : sA3 + 64 * g.C;   // the tail (see below)
  if (TMA) {
    __shared__ uint64_t wbar[2];
    __shared__ int s_fail, wissued[2], wdone[2];
    // the tile's window: rows from tile row - ky - 1 (one period, so in [0, per)),
    // columns from the aligned first column (wrapped, so in [0, W))
    const int per = (g.boundary == HAAR_BOUNDARY_SPHERE) ? 2 * g.H : g.H;
    int yw = (tr * g.T - pr.ky - 1) % per;
    if (yw < 0) yw += per;
    const int xw = (tc * g.T - pr.kx - 1 - o) & Wm;
#pragma unroll
    for (int r = 0; r < 8; ++r) off[r] = tr8_win_off(8 * by, bx) + r * kTr8BoxCols;   // band by
    off[8] = tr8_win_off(8 * by + 8, bx);                                               // first row of band by + 1
    if (threadIdx.x == 0) {
      s_fail = 0;
      wdone[0] = wdone[1] = 0;
      wissued[0] = wissued[1] = 0;
      tc::mbar_init(tc::smem_u32(&wbar[0]), 1);
      tc::mbar_init(tc::smem_u32(&wbar[1]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      for (int c = 0; c < NB && c < g.C; ++c) {
        tr8_issue(win + c * kTr8WinFloats, &mapP, &mapR, xw, yw, c, tc::smem_u32(&wbar[c]));
        wissued[c] = 1;
      }
    }
    __syncthreads();
    switch (o) {
      case 0: tr8_channels_tma<0, NB>(a, pr, s, off, i0, j0, sA3, win, wbar, wissued, wdone, &mapP, &mapR, xw, yw, &s_fail); break;
      case 1: tr8_channels_tma<1, NB>(a, pr, s, off, i0, j0, sA3, win, wbar, wissued, wdone, &mapP, &mapR, xw, yw, &s_fail); break;
      case 2: tr8_channels_tma<2, NB>(a, pr, s, off, i0, j0, sA3, win, wbar, wissued, wdone, &mapP, &mapR, xw, yw, &s_fail); break;
      default: tr8_channels_tma<3, NB>(a, pr, s, off, i0, j0, sA3, win, wbar, wissued, wdone, &mapP, &mapR, xw, yw, &s_fail); break;
    }
    if (s_fail) {
      // a window never arrived: let any copy still in flight land (bounded)
      // before the CTA's shared memory is released, then leave (the status
      // word says why)
      if (threadIdx.x == 0)
        for (int b2 = 0; b2 < NB; ++b2)
          if (wissued[b2] > wdone[b2]) tr8_wait(tc::smem_u32(&wbar[b2]), (uint32_t)(wdone[b2] & 1), nullptr);
      __syncthreads();
      return;
    }
  } else {
    switch (o) {
      case 0: tr8_channels<0>(a, pr, s, off, wrap, i0, j0, sA3); break;
      case 1: tr8_channels<1>(a, pr, s, off, wrap, i0, j0, sA3); break;
      case 2: tr8_channels<2>(a, pr, s, off, wrap, i0, j0, sA3); break;
      default: tr8_channels<3>(a, pr, s, off, wrap, i0, j0, sA3); break;
    }
  }
  pdl_trigger();
  // the tail (levels 4-6, the coarse pass): in the window's shared memory
  // when it fits (every window has been read: the last barrier of the
  // channel loop), else after the level-3 means
  if (TMA) sA4 += a.tail_off;
  float* sA5 = sA4 + 16 * g.C;
  float* sA6 = sA5 + 4 * g.C;
  __syncthreads();
  tr8_level(a, pr, s, 4, 4, sA3, sA4, tr, tc);
  __syncthreads();
  tr8_level(a, pr, s, 5, 2, sA4, sA5, tr, tc);
  __syncthreads();
  tr8_level(a, pr, s, 6, 1, sA5, sA6, tr, tc);
  __syncthreads();
  for (int c = threadIdx.x; c < g.C; c += blockDim.x) {
    if (a.means != nullptr)
      a.means[((long long)s * g.C + c) * g.n_tiles + tile] = sA6[c];
    else  // forward transform: stash the tile mean in the coarse region of the output
      reinterpret_cast<float*>(a.out)[(long long)s * a.st_s + (long long)c * a.st_c + tile] = sA6[c];
  }
  if (a.counters == nullptr) return;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(a.counters + s, 1u);
    s_last = (t == (unsigned)(g.n_tiles - 1)) ? 1 : 0;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float* img = sA6 + ((g.C + 3) & ~3);
  float* img2 = img + ((g.n_tiles + 3) & ~3);
  for (int c = 0; c < g.C; ++c) {
    gather_means(img, a.means + ((long long)s * g.C + c) * g.n_tiles, (int)g.n_tiles, threadIdx.x, blockDim.x);
    coarse_levels<HAAR_OUT_F32>(a, &s_prm, s, c, img, img2);
  }
  if (threadIdx.x == 0) a.counters[s] = 0u;
}

// Coefficient-major translation kernel: one CTA takes a 16 x 16 output tile
// for a group of up to kKscPlanes (shift, channel) planes, one thread per
// (plane, 4 x 4 block).  Levels 1-4 of every plane are staged in shared
// memory as [coefficient][plane] and leave as whole rows of the KSC output
// (the group's consecutive floats of each coefficient), so the stores are
// coalesced instead of one float per 32-byte sector.  The tile means go to
// the workspace; the last tile of a plane group runs the coarse levels of
// all its planes at once (16 threads per plane).
constexpr int kKscPlanes = 48;

// shared floats per plane in the coarse pass: the tile-mean image and the
// scratch image of the next two levels, each rounded to whole float4
__host__ __device__ __forceinline__ int ksc_plane_floats(long long n_tiles) {
  return (int)(((n_tiles + 3) & ~3LL) + ((n_tiles / 16 + 4) & ~3LL));
}

__device__ __forceinline__ int ksc_global_k(const Geometry& g, int kl, int tr, int tc) {
  int lvl, b, r, col;
  if (kl < 192) { lvl = 1; b = kl >> 6; r = (kl >> 3) & 7; col = kl & 7; }
  else if (kl < 240) { lvl = 2; const int k2 = kl - 192; b = k2 >> 4; r = (k2 >> 2) & 3; col = k2 & 3; }
  else if (kl < 252) { lvl = 3; const int k3 = kl - 240; b = k3 >> 2; r = (k3 >> 1) & 1; col = k3 & 1; }
  else { lvl = 4; b = kl - 252; r = 0; col = 0; }
  const int side = 16 >> lvl;
  const int gl = g.q << (2 * (g.n - lvl));
  return gl * (1 + b) + (tr * side + r) * (g.W >> lvl) + tc * side + col;
}

template <int NP>
__global__ void __launch_bounds__(16 * NP) k_shift_ksc(ShiftArgs a, int P) {
  constexpr int kPitch = NP + 1;                // staging row pitch (bank spread)
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_last;
  const Geometry& g = a.g;                      // T = 16, Lt = 4
  const int tile = blockIdx.x;
  const int tr = tile / g.tiles_c, tc = tile - tr * g.tiles_c;
  const int p0 = blockIdx.y * NP;
  const int PG = min(NP, P - p0);
  const int t = threadIdx.x;
  const int pl = t >> 4, blk = t & 15, lane = t & 31;
  const bool on = pl < PG;
  const int plane = p0 + (on ? pl : PG - 1);
  const int s = plane / g.C, c = plane - s * g.C;
  const ShiftParam* pp = a.prm + s;
  pdl_wait();
  const ShiftParam pr = *pp;
  const int by = morton_y(blk), bx = morton_x(blk);
  const int i0 = tr * 16 + 4 * by, j0 = tc * 16 + 4 * bx;
  const int Wm = g.W - 1;
  float* stage = smem;                          // [255][kPitch]

  // resample (translation: 5 x 8 aligned window, pre-scaled by 1/2) and levels 1-2
  const int o = (-(pr.kx + 1)) & 3;
  const float* F = a.pix + (long long)c * g.N;
  float4 v[5][2];
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    int i = i0 - pr.ky - 1 + r, sh = 0;
    if (g.boundary == HAAR_BOUNDARY_TORUS) {
      i &= (g.H - 1);
    } else {
#pragma unroll 1
      for (int it = 0; it < 8 && (i < 0 || i >= g.H); ++it) {
        i = (i < 0) ? -1 - i : 2 * g.H - 1 - i;
        sh ^= 1;
      }
    }
    const int ca = j0 - pr.kx - 1 + (sh ? (g.W >> 1) : 0) - o;
    v[r][0] = __ldg(reinterpret_cast<const float4*>(F + i * g.W + (ca & Wm)));
    v[r][1] = __ldg(reinterpret_cast<const float4*>(F + i * g.W + ((ca + 4) & Wm)));
  }
  float x[16];
  const float wy0 = 0.5f * pr.wy0, wy1 = 0.5f * pr.wy1;
  switch (o) {
    case 0: bilin_tr<0>(v, pr.wx0, pr.wx1, wy0, wy1, x); break;
    case 1: bilin_tr<1>(v, pr.wx0, pr.wx1, wy0, wy1, x); break;
    case 2: bilin_tr<2>(v, pr.wx0, pr.wx1, wy0, wy1, x); break;
    default: bilin_tr<3>(v, pr.wx0, pr.wx1, wy0, wy1, x); break;
  }
  const unsigned pm = pr.perm_mask;
  float A1[4];
#pragma unroll
  for (int sa = 0; sa < 2; ++sa)
#pragma unroll
    for (int sc = 0; sc < 2; ++sc) {
      const float ea = x[(2 * sa) * 4 + 2 * sc], eb = x[(2 * sa) * 4 + 2 * sc + 1];
      const float ec = x[(2 * sa + 1) * 4 + 2 * sc], ed = x[(2 * sa + 1) * 4 + 2 * sc + 1];
      A1[2 * sa + sc] = (ea + eb) + (ec + ed);
      const float d[3] = {(eb + ed) - (ea + ec), (ec + ed) - (ea + eb), (ea + ed) - (eb + ec)};
      const int r = 2 * by + sa, col = 2 * bx + sc;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        float val = d[b];
        if (pm & 2u) val = perm_value(a, pr, c, 1, b, tr * 8 + r, tc * 8 + col);
        if (on) stage[(b * 64 + r * 8 + col) * kPitch + pl] = val;
      }
    }
  float A;
  {
    const float ea = A1[0], eb = A1[1], ec = A1[2], ed = A1[3];
    const float d[3] = {0.5f * ((eb + ed) - (ea + ec)), 0.5f * ((ec + ed) - (ea + eb)), 0.5f * ((ea + ed) - (eb + ec))};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      float val = d[b];
      if (pm & 4u) val = perm_value(a, pr, c, 2, b, tr * 4 + by, tc * 4 + bx);
      if (on) stage[(192 + b * 16 + by * 4 + bx) * kPitch + pl] = val;
    }
    A = 0.5f * ((ea + eb) + (ec + ed));
  }
  // levels 3 and 4 within the plane's 16 lanes (Morton order: strides 1, 4)
#pragma unroll
  for (int step = 0; step < 2; ++step) {
    const int st = step ? 4 : 1, lvl = 3 + step;
    const int base = lane & ~(4 * st - 1);
    const float e0 = __shfl_sync(0xffffffffu, A, base);
    const float e1 = __shfl_sync(0xffffffffu, A, base + st);
    const float e2 = __shfl_sync(0xffffffffu, A, base + 2 * st);
    const float e3 = __shfl_sync(0xffffffffu, A, base + 3 * st);
    const int m = (lane - base) >> (2 * step);
    if ((lane & (st - 1)) == 0 && m < 3) {
      float val = (m == 0) ? 0.5f * ((e1 + e3) - (e0 + e2))
                : (m == 1) ? 0.5f * ((e2 + e3) - (e0 + e1)) : 0.5f * ((e0 + e3) - (e1 + e2));
      const int rr = by >> (lvl - 2), cc = bx >> (lvl - 2);
      if ((pm >> lvl) & 1u) val = perm_value(a, pr, c, lvl, m, tr * (16 >> lvl) + rr, tc * (16 >> lvl) + cc);
      const int kl = (lvl == 3) ? 240 + m * 4 + rr * 2 + cc : 252 + m;
      if (on) stage[kl * kPitch + pl] = val;
    }
    A = 0.5f * ((e0 + e1) + (e2 + e3));
  }
  if (blk == 0 && on) {
    a.means[(long long)plane * g.n_tiles + tile] = A;
    __threadfence();
  }
  __syncthreads();

  // rows of the group's PG consecutive floats, one coefficient per warp at a time
  float* out = reinterpret_cast<float*>(a.out);
  for (int kl = t >> 5; kl < 255; kl += blockDim.x >> 5) {
    const int k = ksc_global_k(g, kl, tr, tc);                // warp-uniform
    if (k < a.K) {
      float* orow = out + (long long)k * P + p0;
      const float* srow = stage + kl * kPitch;
      for (int q = lane; q < PG; q += 32) orow[q] = srow[q];
    }
  }

  pdl_trigger();                                  // the tile's rows are written
  // the tile means were published (stores + fence by their writers) before
  // the barrier above; thread 0 counts the tile and, last, acquires them all
  if (t == 0) {
    const unsigned n = atomicAdd(a.counters + blockIdx.y, 1u);
    s_last = (n == (unsigned)(g.n_tiles - 1)) ? 1 : 0;
    if (s_last) __threadfence();
  }
  __syncthreads();
  if (!s_last) return;
  // coarse levels of every plane of the group, 16 threads per plane; both
  // images start on 16-byte boundaries (the passes read them as float4)
  const int nt4 = (g.n_tiles + 3) & ~3;
  const int per = ksc_plane_floats(g.n_tiles);
  float* img = smem + pl * per;
  float* img2 = img + nt4;
  if (on) gather_means(img, a.means + (long long)plane * g.n_tiles, (int)g.n_tiles, blk, 16);
  // threads of absent planes (partial group) take part in the barriers only
  coarse_levels_t<HAAR_OUT_F32, false>(a, pp, s, c, img, img2, on ? blk : (1 << 30), 16);
  if (t == 0) a.counters[blockIdx.y] = 0u;
}

// Coarse levels of the forward transform, in place: one CTA per map.
__global__ void __launch_bounds__(kThreads) k_coarse_inplace(ShiftArgs a) {
  extern __shared__ __align__(16) float smem[];
  const int s = blockIdx.x;
  float* out = reinterpret_cast<float*>(a.out) + (long long)s * a.st_s;
  float* img = smem;
  float* img2 = smem + ((a.g.n_tiles + 3) & ~3);   // float4-aligned
  for (int t = threadIdx.x; t < a.g.n_tiles; t += blockDim.x) img[t] = out[t];
  __syncthreads();
  // put() multiplies by a.scale; the tile means were stored unscaled
  coarse_levels<HAAR_OUT_F32>(a, nullptr, s, 0, img, img2);
}

// Per-launch set-up: blocks [0, nbp) synthesise the pixel map from the
// coefficients (inverse transform, one thread per pixel summing its
// ancestors; for the rotation kinds one thread per texel of the interleaved
// map, see pix_floats()).  Translations and the chain-rule route: the last
// block builds the shift records in FP64 and clears the per-shift tile
// counters.  Rotations: block nbp + s builds rotation s's record and its
// tables in FP64 (the one-time construction of the shift's mixing weights).
struct SetupArgs {
  int H, W, C, n, q, kind, boundary, S, nbp;
  long long cin_stride;   // floats between input channels (the full map's N)
  double pscale;          // translation scale (2^-start_level)
  const float* cin;
  float* pix;
  const double* params;
  ShiftParam* prm;
  unsigned* counters;
  const float4* trig;     // rotations: the map's pair tables, rows [H] then columns [W]
  float4* rtab;           // rotations: per-rotation tables
  long long rt_stride;
  float* pixE;            // translations: synthesise the extended map [C][HE][WE] instead of pix
  int HE, WE;
};

__device__ __forceinline__ float synth_pixel(const float* cf, int i, int j, int W, int n, int q) {
  float x = __ldg(cf + (j >> n));
  for (int l = n; l >= 1; --l) {
    const int r = i >> l, cc = j >> l;
    const int qi = (i >> (l - 1)) & 1, qj = (j >> (l - 1)) & 1;
    const long long gl = (long long)q << (2 * (n - l));
    const long long o = (long long)r * (W >> l) + cc;
    const float hv = __ldg(cf + gl + o), vv = __ldg(cf + 2 * gl + o), dv = __ldg(cf + 3 * gl + o);
    x = 0.5f * (x + (qj ? hv : -hv) + (qi ? vv : -vv) + ((qi == qj) ? dv : -dv));
  }
  return x;
}

__device__ __forceinline__ float4 split2(double s, double c) {
  const float sh = (float)s, ch = (float)c;
  return make_float4(sh, (float)(s - (double)sh), ch, (float)(c - (double)ch));
}

__device__ void rotation_matrix(const SetupArgs& a, int s, double R[9]) {
  if (a.kind == HAAR_SHIFT_ROTATE) {
    for (int k = 0; k < 9; ++k) R[k] = a.params[9 * s + k];
    return;
  }
  const double al = a.params[3 * s], be = a.params[3 * s + 1], ga = a.params[3 * s + 2];
  const double ca = cos(al), sa = sin(al), cb = cos(be), sb = sin(be);
  const double cg = cos(ga), sg = sin(ga);
  const double Rx[9] = {1, 0, 0, 0, ca, -sa, 0, sa, ca};
  const double Ry[9] = {cb, 0, sb, 0, 1, 0, -sb, 0, cb};
  const double Rz[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1};
  double M[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      M[3 * r + c] = Ry[3 * r] * Rx[c] + Ry[3 * r + 1] * Rx[3 + c] + Ry[3 * r + 2] * Rx[6 + c];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = Rz[3 * r] * M[c] + Rz[3 * r + 1] * M[3 + c] + Rz[3 * r + 2] * M[6 + c];
}

__global__ void __launch_bounds__(kThreads) k_setup(SetupArgs a) {
  pdl_trigger();                                  // the shift kernel may be scheduled (it waits for this grid)
  const long long N = (long long)a.H * a.W;
  const bool rot = a.kind == HAAR_SHIFT_ROTATE || a.kind == HAAR_SHIFT_ROTATE_EULER;
  if ((int)blockIdx.x < a.nbp) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rot) {
      // texel (group g, row i, column j): channels 3g..3g+2 at columns j and j+1
      const int G = (a.C + 2) / 3;
      if (e >= N * G) return;
      const int gi = (int)(e / N);
      const long long rem = e - (long long)gi * N;
      const int i = (int)(rem / a.W), j = (int)(rem - (long long)i * a.W), j1 = (j + 1) & (a.W - 1);
      float v[6];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int c = 3 * gi + t;
        if (c < a.C) {
          const float* cf = a.cin + (long long)c * a.cin_stride;
          v[2 * t] = synth_pixel(cf, i, j, a.W, a.n, a.q);
          v[2 * t + 1] = synth_pixel(cf, i, j1, a.W, a.n, a.q);
        } else {
          v[2 * t] = v[2 * t + 1] = 0.0f;
        }
      }
      float4* o = reinterpret_cast<float4*>(a.pix) + 2 * e;
      o[0] = make_float4(v[0], v[1], v[2], v[3]);
      o[1] = make_float4(v[4], v[5], 0.0f, 0.0f);
      return;
    }
    if (a.pixE != nullptr) {
      // the extended map: each synthesised pixel (i, j) goes to every place it
      // appears there.  Extended rows: one period (SPHERE: the map's rows,
      // then the rows mirrored across the pole half a turn round; TORUS: the
      // map's rows) and its first 65 rows again; extended columns: the map's
      // columns and its first 68 again.
      if (e >= N * a.C) return;
      const int c = (int)(e / N);
      const long long rem = e - (long long)c * N;
      const int i = (int)(rem / a.W), j = (int)(rem - (long long)i * a.W);
      const float v = synth_pixel(a.cin + (long long)c * a.cin_stride, i, j, a.W, a.n, a.q);
      float* E = a.pixE + (long long)c * a.HE * a.WE;
      const bool sph = a.boundary == HAAR_BOUNDARY_SPHERE;
      const int per = sph ? 2 * a.H : a.H;
      // rows i + k per, columns j + m W (and, SPHERE, the mirrored rows
      // 2H - 1 - i + k per at column (j - W/2) mod W + m W)
#pragma unroll 1
      for (int mir = 0; mir < (sph ? 2 : 1); ++mir) {
        const int ei0 = mir ? 2 * a.H - 1 - i : i;
        const int ej0 = mir ? (j - (a.W >> 1)) & (a.W - 1) : j;
        for (int ei = ei0; ei < a.HE; ei += per)
          for (int ej = ej0; ej < a.WE; ej += a.W) E[(long long)ei * a.WE + ej] = v;
      }
      return;
    }
    if (e >= N * a.C) return;
    const int c = (int)(e / N);
    const long long rem = e - (long long)c * N;
    const int i = (int)(rem / a.W), j = (int)(rem - (long long)i * a.W);
    a.pix[e] = synth_pixel(a.cin + (long long)c * a.cin_stride, i, j, a.W, a.n, a.q);
    return;
  }
  if (rot) {
    // rotations, one warp each (8 per block): lane 0 finds R = Ry(a) Rx(b)
    // Ry(c) (proper Euler angles) in FP64 and writes the record; the warp
    // then builds the rotation's float-pair tables
    __shared__ double sh[8][6];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = (blockIdx.x - a.nbp) * 8 + w;
    if (s >= a.S) return;
    if (lane == 0) {
      double R[9];
      rotation_matrix(a, s, R);
      yxy_angles(R, sh[w]);
      ShiftParam p;
      p.kx = p.ky = 0;
      p.wx0 = p.wy0 = 1.0f;
      p.wx1 = p.wy1 = 0.0f;
      p.perm_mask = 0u;
      p.order = 0;
      for (int k = 0; k < 9; ++k) p.R[k] = (float)R[k];
      p.a_px = (float)(atan2(sh[w][0], sh[w][1]) * (a.W / (2.0 * 3.14159265358979323846)) - 0.5);
      p.pad2[0] = p.pad2[1] = 0.0f;
      a.prm[s] = p;
      a.counters[s] = 0u;
    }
    __syncwarp();
    const RotAngles g = rot_angles(sh[w]);
    float4* rt = a.rtab + (long long)s * a.rt_stride;
    for (int j = lane; j < a.W; j += 32) rot_col_entries(a.trig[a.H + j], g, rt[j], rt[a.W + j]);
    for (int i = lane; i < a.H; i += 32) rot_row_entries(a.trig[i], g, rt[2 * a.W + 2 * i], rt[2 * a.W + 2 * i + 1]);
    return;
  }
  for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
    ShiftParam p;
    p.kx = p.ky = 0;
    p.wx0 = p.wy0 = 1.0f;
    p.wx1 = p.wy1 = 0.0f;
    p.perm_mask = 0u;
    p.order = 0;
    for (int k = 0; k < 9; ++k) p.R[k] = (k % 4 == 0) ? 1.0f : 0.0f;
    p.a_px = 0.0f;
    p.pad2[0] = p.pad2[1] = 0.0f;
    if (a.kind == HAAR_SHIFT_TRANSLATE) {
      const double dx = a.params[2 * s] * a.pscale, dy = a.params[2 * s + 1] * a.pscale;
      const double W = a.W;
      const double per = (a.boundary == HAAR_BOUNDARY_SPHERE) ? 2.0 * a.H : (double)a.H;
      double x = dx - W * floor(dx / W);
      if (x >= W) x -= W;
      if (!(x >= 0.0 && x < W)) x = 0.0;     // non-finite or rounding outside [0, W)
      double y = dy - per * floor(dy / per);
      if (y >= per) y -= per;
      if (!(y >= 0.0 && y < per)) y = 0.0;
      const double fx = floor(x), fy = floor(y);
      const double tx = x - fx, ty = y - fy;
      p.kx = (int)fx;
      p.ky = (int)fy;
      p.wx0 = (float)(1.0 - tx);
      p.wx1 = (float)tx;
      p.wy0 = (float)(1.0 - ty);
      p.wy1 = (float)ty;
      if (tx == 0.0 && ty == 0.0) {
        for (int l = 1; l <= a.n + 1; ++l) {
          const int B = 1 << (l > a.n ? a.n : l);
          const bool crosses = (a.boundary == HAAR_BOUNDARY_SPHERE) && p.ky != 0;
          if (p.kx % B == 0 && p.ky % B == 0 && (!crosses || ((a.W / 2) % B) == 0))
            p.perm_mask |= 1u << l;
        }
      }
    } else {
      double R[9];
      rotation_matrix(a, s, R);
      for (int k = 0; k < 9; ++k) p.R[k] = (float)R[k];
    }
    a.prm[s] = p;
    a.counters[s] = 0u;
  }
  if (a.kind != HAAR_SHIFT_TRANSLATE) return;
  // translations: list the shifts grouped by column phase (kx + 1) mod 4 in
  // the records' `order` fields, so that the batch kernel's co-resident CTAs
  // mostly run the same one of its four phase-specialised code paths
  __shared__ int cnt[4];
  if (threadIdx.x < 4) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < a.S; s += blockDim.x) atomicAdd(&cnt[(-(a.prm[s].kx + 1)) & 3], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int o = 0; o < 4; ++o) {
      const int c = cnt[o];
      cnt[o] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < a.S; s += blockDim.x) {
    const int pos = atomicAdd(&cnt[(-(a.prm[s].kx + 1)) & 3], 1);
    a.prm[pos].order = s;
  }
}

// Rotation tables of the map (see trig_floats()): pixel-centre sines and
// cosines in FP64, kept as float pairs.
__global__ void k_trig(int H, int W, float* trig) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const double pi = 3.14159265358979323846;
  float4* t = reinterpret_cast<float4*>(trig);
  if (e < H) {
    const double x = (e + 0.5) * pi / H;
    t[e] = split2(sin(x), cos(x));
  } else if (e < H + W) {
    const int j = e - H;
    const double x = (j + 0.5) * 2.0 * pi / W;
    t[H + j] = split2(sin(x), cos(x));
  }
}

__global__ void __launch_bounds__(kThreads) k_inverse(int H, int W, int n, int q, long long total,
                                                      const float* cin, float* maps) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const long long N = (long long)H * W;
  const long long b = e / N;
  const long long rem = e - b * N;
  const int i = (int)(rem / W), j = (int)(rem - (long long)i * W);
  maps[e] = synth_pixel(cin + b * N, i, j, W, n, q);
}

// ------------------------------------------------------------------ launchers

static size_t shift_smem_bytes(const Geometry& g, int kind) {
  const int CG = (kind == KIND_ROTATE) ? kRotChannels : 1;
  const int win = (kind == KIND_TRANSLATE) ? (g.T + 1) * (g.T + 1) : 0;
  const int winr = (win + 3) & ~3;
  size_t pix = (size_t)CG * g.T * g.T;
  const size_t coarse = (size_t)g.n_tiles + (size_t)g.n_tiles / 4 + 8;
  if (pix < coarse) pix = coarse;
  const size_t scratch = (size_t)(g.T / 4) * (g.T / 4) + 8 + g.T;
  return sizeof(float) * ((size_t)winr + pix + scratch);
}

template <int KIND, int OUT, int CG>
static haar_status_t launch_reg(const ShiftArgs& a0, int S, cudaStream_t st) {
  ShiftArgs a = a0;
  const int nb = a.g.T / 4;
  // shared floats: the group values sA [CG][nb^2 / 16], then (last CTA of a
  // shift) the tile-mean image and its scratch, each float4-aligned; for
  // rotations of maps with W + H <= 1536, the two coordinate tables after them
  const size_t sa = ((size_t)CG * nb * nb / 16 + 3) & ~(size_t)3;
  const size_t nt4 = ((size_t)a.g.n_tiles + 3) & ~(size_t)3;
  const size_t fl = (sa + nt4 + (size_t)a.g.n_tiles / 4 + 16 + 3) & ~(size_t)3;
  const bool smt = KIND == KIND_ROTATE && a.g.W + a.g.H <= 1536;
  const size_t sm = (fl + (smt ? 4 * (size_t)(a.g.W + a.g.H) : 0)) * sizeof(float);
  a.tab_off = (int)fl;
  auto fr = smt ? k_shift_reg<KIND, OUT, CG, true> : k_shift_reg<KIND, OUT, CG, false>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_shift_reg)");
  }
  dim3 grid(a.g.n_tiles, S, (a.g.C + CG - 1) / CG);
  return cuda_check(launch_pdl(fr, grid, dim3(nb * nb), sm, st, a), "k_shift_reg launch");
}

// Channels per thread: a rotation shares its coordinates across kRotChannels
// channels; a translation shares only its window addresses, so it takes
// kRotChannels channels per thread only when that still leaves several
// waves of CTAs (otherwise one channel per CTA, for parallelism).
// The 8 x 8-block translation kernel serves F32 batches of many shifts into a
// k-contiguous, untruncated layout with 16-byte aligned planes.
static bool tr8_eligible(const ShiftArgs& a, int S) {
  return a.g.T == 64 && a.st_k == 1 && a.scale == 1.0f && a.K >= a.g.N && a.st_s % 4 == 0 && a.st_c % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(a.out) & 15) == 0 && (long long)a.g.n_tiles * S >= 2432;
}

static haar_status_t launch_tr8(const ShiftArgs& a0, int S, cudaStream_t st) {
  ShiftArgs a = a0;
  const bool tma = a.pixE != nullptr;
  const bool tail_win = tr8_tail_in_window(tma, a.g.C, a.g.n_tiles);
  a.tail_off = tail_win ? 0 : (tma ? kTr8Windows * kTr8WinFloats : 0) + 64 * a.g.C;
  // [window (TMA-fed form; + 32 for its 128-byte alignment) | level-3 means
  // [C][64] | the tail, unless it sits in the window]
  const size_t fl = (tma ? kTr8Windows * (size_t)kTr8WinFloats + 32 : 0) + 64 * (size_t)a.g.C +
                    (tail_win ? 0 : (size_t)tr8_tail_floats(a.g.C, a.g.n_tiles));
  const size_t sm = ((fl + 3) & ~(size_t)3) * sizeof(float);
  CUtensorMap mapP, mapR;            // the window's 72 x 8 bands and its 72 x 1 last row
  memset(&mapP, 0, sizeof(mapP));
  memset(&mapR, 0, sizeof(mapR));
  if (tma && (!encode_3d_f32(&mapP, a.pixE, (uint64_t)a.WE, (uint64_t)a.HE, (uint64_t)a.g.C, kTr8BoxCols,
                             kTr8BandRows) ||
              !encode_3d_f32(&mapR, a.pixE, (uint64_t)a.WE, (uint64_t)a.HE, (uint64_t)a.g.C, kTr8BoxCols, 1)))
    return set_error(HAAR_ERR_CUDA, "haar_shift: cuTensorMapEncodeTiled (extended map) failed");
  auto fn = tma ? k_shift_tr8<true, kTr8Windows> : k_shift_tr8<false, kTr8Windows>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_shift_tr8)");
  }
  return cuda_check(launch_pdl(fn, dim3(a.g.n_tiles, S), dim3(kTr8Threads), sm, st, a, mapP, mapR),
                    "k_shift_tr8 launch");
}

bool tr8_tma_plan(const haar_shift_desc_t& d, const Geometry& g, int K, int max_shifts) {
  return d.kind == HAAR_SHIFT_TRANSLATE && d.out_type == HAAR_OUT_F32 && d.out_layout == HAAR_LAYOUT_SCK &&
         g.T == 64 && K >= g.N && g.H >= 64 && (long long)g.n_tiles * max_shifts >= 2432;
}

// this launch runs the TMA-fed batch kernel (the set-up then synthesises the
// extended map instead of the plain one)
static bool tr8_tma_use(const haar_shift_plan_s* p, int S, const void* out) {
  return p->pixE != nullptr && p->desc.kind == HAAR_SHIFT_TRANSLATE && (long long)p->geo.n_tiles * S >= 2432 &&
         (reinterpret_cast<uintptr_t>(out) & 15) == 0;
}

template <int KIND, int OUT>
static haar_status_t launch_k(const ShiftArgs& a, int S, cudaStream_t st) {
  if constexpr (KIND == KIND_TRANSLATE && OUT == HAAR_OUT_F32) {
    if (tr8_eligible(a, S)) return launch_tr8(a, S, st);
  }
  if (a.g.T >= 32) {
    if constexpr (KIND == KIND_COPY) {
      return launch_reg<KIND, OUT, 1>(a, S, st);
    } else if constexpr (KIND == KIND_ROTATE) {
      return launch_reg<KIND, OUT, kRotChannels>(a, S, st);
    } else {
      if ((long long)a.g.n_tiles * S >= 2432) return launch_reg<KIND, OUT, kRotChannels>(a, S, st);
      return launch_reg<KIND, OUT, 1>(a, S, st);
    }
  }
  const int CG = (KIND == KIND_ROTATE) ? kRotChannels : 1;
  const size_t sm = shift_smem_bytes(a.g, KIND);
  auto fn = k_shift<KIND, OUT>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_shift)");
  }
  dim3 grid(a.g.n_tiles, S, (a.g.C + CG - 1) / CG);
  return cuda_check(launch_pdl(fn, grid, dim3(kThreads), sm, st, a), "k_shift launch");
}

template <int KIND>
static haar_status_t launch_out(const ShiftArgs& a, int out_type, int S, cudaStream_t st) {
  switch (out_type) {
    case HAAR_OUT_F32: return launch_k<KIND, HAAR_OUT_F32>(a, S, st);
    case HAAR_OUT_BF16_HILO: return launch_k<KIND, HAAR_OUT_BF16_HILO>(a, S, st);
    default: return launch_k<KIND, HAAR_OUT_F16>(a, S, st);
  }
}

haar_status_t launch_trig(haar_shift_plan_s* p, cudaStream_t st) {
  const int tot = p->geo.H + p->geo.W;
  k_trig<<<(tot + 255) / 256, 256, 0, st>>>(p->geo.H, p->geo.W, p->trig);
  return cuda_check(cudaGetLastError(), "k_trig launch");
}

haar_status_t launch_setup(haar_shift_plan_s* p, const float* coeffs_in, const double* params, const void* out,
                           int S, cudaStream_t st) {
  SetupArgs a;
  const Geometry& g = p->geo;
  a.H = g.H; a.W = g.W; a.C = g.C; a.n = g.n; a.q = g.q;
  a.kind = p->desc.kind;
  a.boundary = g.boundary;
  a.S = S;
  const bool rot = a.kind == HAAR_SHIFT_ROTATE || a.kind == HAAR_SHIFT_ROTATE_EULER;
  const bool ext = tr8_tma_use(p, S, out);
  a.pixE = ext ? p->pixE : nullptr;
  a.HE = p->pixE_H;
  a.WE = p->pixE_W;
  const long long total = rot ? g.N * ((g.C + 2) / 3) : g.N * g.C;
  a.nbp = (int)((total + kThreads - 1) / kThreads);
  a.cin = coeffs_in;
  a.cin_stride = p->cin_stride;
  a.pscale = p->pscale;
  a.pix = p->pix;
  a.params = params;
  a.prm = p->prm;
  a.counters = p->counters;
  a.trig = reinterpret_cast<const float4*>(p->trig);
  a.rtab = reinterpret_cast<float4*>(p->rtab);
  a.rt_stride = rot_table_float4s(g.H, g.W);
  if (rot && p->rtab == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "rotation tables missing");
  k_setup<<<a.nbp + (rot ? (S + 7) / 8 : 1), kThreads, 0, st>>>(a);
  return cuda_check(cudaGetLastError(), "k_setup launch");
}

// The coefficient-major kernel serves F32 KSC translations whose tile-mean
// workspace and shared-memory coarse pass fit.
bool ksc_eligible(const haar_shift_desc_t& d, const Geometry& g, int S) {
  if (d.kind != HAAR_SHIFT_TRANSLATE || d.out_type != HAAR_OUT_F32 || d.out_layout != HAAR_LAYOUT_KSC) return false;
  if (g.H < 16) return false;
  const long long P = (long long)S * g.C;
  if ((P + kKscPlanes - 1) / kKscPlanes > S) return false;                 // one counter per plane group
  const long long n16 = (long long)(g.H / 16) * (g.W / 16);
  return ksc_smem_floats(n16, kKscPlanes) * sizeof(float) <= 200 * 1024;
}

// Planes per CTA: 48, or 24 when a 48-plane grid would not fill two CTAs per
// SM (e.g. the 16 RGB shifts of a 128 x 256 map: 128 tiles) and the plane
// groups still fit the per-shift counters.
static int ksc_planes(const Geometry& g16, long long P, int S) {
  const long long g48 = (P + kKscPlanes - 1) / kKscPlanes, g24 = (P + 23) / 24;
  return ((long long)g16.n_tiles * g48 < 304 && g24 <= S) ? 24 : kKscPlanes;
}

size_t ksc_means_floats(const Geometry& g, int S) {
  return (size_t)S * g.C * (size_t)(g.H / 16) * (g.W / 16);
}

size_t ksc_smem_floats(long long n16, int planes) {
  const long long coarse = (long long)planes * ksc_plane_floats(n16);
  const long long stage = 255LL * (planes + 1);
  return (size_t)(coarse > stage ? coarse : stage);
}

static haar_status_t launch_ksc(haar_shift_plan_s* p, const float* coeffs_in, int S, void* out, cudaStream_t st) {
  ShiftArgs a;
  const Geometry g = make_geometry(p->geo.H, p->geo.W, p->geo.C, p->geo.boundary, 16);
  a.g = g;
  a.K = p->K;
  const long long P = (long long)S * g.C;
  a.st_s = g.C; a.st_c = 1; a.st_k = P;
  a.plane = 0;
  a.out = out;
  a.pix = p->pix;
  a.cin = coeffs_in;
  a.cin_stride = p->cin_stride;
  a.prm = p->prm;
  a.means = p->means;
  a.counters = p->counters;
  a.rows = nullptr;
  a.rtab = nullptr;
  a.rt_stride = 0;
  a.tab_off = 0;
  a.scale = 1.0f;
  a.u_scale = a.v_scale = 0.0f;
  const int np = ksc_planes(g, P, S);
  const size_t sm = ksc_smem_floats(g.n_tiles, np) * sizeof(float);
  auto fn = (np == 24) ? k_shift_ksc<24> : k_shift_ksc<kKscPlanes>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_shift_ksc)");
  }
  dim3 grid(g.n_tiles, (unsigned)((P + np - 1) / np));
  return cuda_check(launch_pdl(fn, grid, dim3(16 * np), sm, st, a, (int)P), "k_shift_ksc launch");
}

haar_status_t launch_shift(haar_shift_plan_s* p, const float* coeffs_in, int S, void* out,
                           cudaStream_t st) {
  if (ksc_eligible(p->desc, p->geo, S) && ksc_means_floats(p->geo, S) <= p->means_cap)
    return launch_ksc(p, coeffs_in, S, out, st);
  ShiftArgs a;
  const Geometry& g = p->geo;
  a.g = g;
  a.K = p->K;
  const long long K = p->K, C = g.C;
  switch (p->desc.out_layout) {
    case HAAR_LAYOUT_SCK: a.st_s = C * K; a.st_c = K; a.st_k = 1; break;
    case HAAR_LAYOUT_SKC: a.st_s = K * C; a.st_c = 1; a.st_k = C; break;
    case HAAR_LAYOUT_SKC4: a.st_s = K * 4; a.st_c = 1; a.st_k = 4; break;
    default: a.st_s = C; a.st_c = 1; a.st_k = (long long)S * C; break;
  }
  a.plane = (long long)S * C * K;
  a.out = out;
  a.pix = p->pix;
  a.cin = coeffs_in;
  a.cin_stride = p->cin_stride;
  a.prm = p->prm;
  a.means = p->means;
  a.counters = p->counters;
  a.rows = reinterpret_cast<const float4*>(p->trig);
  a.rtab = reinterpret_cast<const float4*>(p->rtab);
  a.rt_stride = rot_table_float4s(g.H, g.W);
  a.tab_off = 0;
  a.scale = 1.0f;
  a.u_scale = (float)(g.H / 3.14159265358979323846);
  a.v_scale = (float)(g.W / (2.0 * 3.14159265358979323846));
  a.status = p->status;
  if (tr8_tma_use(p, S, out)) {
    a.pixE = p->pixE;
    a.HE = p->pixE_H;
    a.WE = p->pixE_W;
  }
  if (p->desc.kind == HAAR_SHIFT_TRANSLATE) return launch_out<KIND_TRANSLATE>(a, p->desc.out_type, S, st);
  return launch_out<KIND_ROTATE>(a, p->desc.out_type, S, st);
}

haar_status_t launch_forward(int H, int W, int batch, const float* maps, float* coeffs, float scale,
                             cudaStream_t st) {
  ShiftArgs a;
  a.g = make_geometry(H, W, 1, HAAR_BOUNDARY_SPHERE);
  a.K = H * W;
  a.st_s = (long long)H * W;
  a.st_c = 0;
  a.st_k = 1;
  a.plane = 0;
  a.out = coeffs;
  a.pix = maps;
  a.cin = nullptr;
  a.cin_stride = 0;
  a.prm = nullptr;
  a.means = nullptr;
  a.counters = nullptr;
  a.rows = nullptr;
  a.rtab = nullptr;
  a.rt_stride = 0;
  a.tab_off = 0;
  a.scale = scale;
  a.u_scale = a.v_scale = 0.0f;
  // details are scaled by put(); tile means are stashed unscaled and scaled
  // when k_coarse_inplace writes the coarse levels through put()
  haar_status_t r = launch_k<KIND_COPY, HAAR_OUT_F32>(a, batch, st);
  if (r != HAAR_OK) return r;
  const size_t sm = sizeof(float) * ((size_t)a.g.n_tiles * 2 + 16);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_coarse_inplace, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_coarse_inplace)");
  }
  k_coarse_inplace<<<batch, kThreads, sm, st>>>(a);
  return cuda_check(cudaGetLastError(), "k_coarse_inplace launch");
}

haar_status_t launch_inverse(int H, int W, int batch, const float* coeffs, float* maps,
                             cudaStream_t st) {
  const Geometry g = make_geometry(H, W, 1, HAAR_BOUNDARY_SPHERE);
  const long long total = (long long)batch * g.N;
  const long long nb = (total + kThreads - 1) / kThreads;
  k_inverse<<<(unsigned)nb, kThreads, 0, st>>>(H, W, g.n, g.q, total, coeffs, maps);
  return cuda_check(cudaGetLastError(), "k_inverse launch");
}

}  // namespace hs
