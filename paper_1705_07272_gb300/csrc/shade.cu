// Per-vertex double product on sm_103a (CUDA-core forms): dense FP32
// transport, top-K CSR FP32 transport and view-binned top-K FP16 transport,
// plus the view-bin selection.
//
// The double product is the light-transport integral of Eq. (1)-(3) with the
// BRDF, cosine and visibility folded into one transfer function; for
// orthonormal Haar bases it is the inner product of the two coefficient
// vectors: radiance[v][s][c] = sum_k T[v][k] L'[s][c][k].  Top-K storage is
// the non-linear wavelet approximation cited in Sec. "Haar-domain methods".
#include "common.cuh"
#include "tc.cuh"

namespace hs {

// ---------------------------------------------------------------- dense FP32
// One warp per vertex; lanes stride over k with float4 loads; up to 8 output
// columns (s, c) per pass over the row.
__global__ void __launch_bounds__(256) k_shade_dense_f32(const float* __restrict__ T, int V, int K,
                                                         const float* __restrict__ L, int ldl, int ncols,
                                                         float* __restrict__ R) {
  pdl_wait();                                     // inputs come from the previous kernel
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= V) return;
  const float* t = T + (long long)warp * K;
  const bool vec = ((K & 3) == 0) && ((ldl & 3) == 0);
  for (int c0 = 0; c0 < ncols; c0 += 8) {
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
    if (vec) {
      for (int k = 4 * lane; k < K; k += 128) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(t + k));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (c0 + j < ncols) {
            const float4 l = __ldg(reinterpret_cast<const float4*>(L + (long long)(c0 + j) * ldl + k));
            acc[j] = fmaf(x.x, l.x, fmaf(x.y, l.y, fmaf(x.z, l.z, fmaf(x.w, l.w, acc[j]))));
          }
        }
      }
    } else {
      for (int k = lane; k < K; k += 32) {
        const float x = __ldg(t + k);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < ncols) acc[j] = fmaf(x, __ldg(L + (long long)(c0 + j) * ldl + k), acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float v = acc[j];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[j] = v;
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (c0 + j < ncols) R[(long long)warp * ncols + c0 + j] = acc[j];
    }
  }
}

// ---------------------------------------------------------------- CSR FP32
// Lighting is coefficient-major: L[k][ncols] (ncols = S*C, a multiple of 4),
// so one non-zero gathers one contiguous row.  One warp per vertex: 8 groups
// of 4 lanes take 8 non-zeros at a time, each lane accumulates NQL float4 of
// the row; the groups are reduced with shuffles at the end.
template <int NQL>
__global__ void __launch_bounds__(256) k_shade_csr_f32(const float* __restrict__ vals,
                                                       const uint16_t* __restrict__ idx,
                                                       const int32_t* __restrict__ rowptr, int V,
                                                       const float* __restrict__ L, int NL, int ncols,
                                                       float* __restrict__ R) {
  pdl_wait();                                     // inputs come from the previous kernel
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= V) return;
  const int g = lane >> 2, l4 = lane & 3;
  const int beg = __ldg(rowptr + warp), end = __ldg(rowptr + warp + 1);
  const int nq = ncols >> 2;
  for (int q0 = 0; q0 < nq; q0 += 4 * NQL) {
    float4 acc[NQL];
#pragma unroll
    for (int m = 0; m < NQL; ++m) acc[m] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int j = beg + g; j < end; j += 8) {
      const int k = __ldg(idx + j);
      const float t = (k < NL) ? __ldg(vals + j) : 0.0f;   // out-of-range entries are ignored
      const float4* Lr = reinterpret_cast<const float4*>(L + (long long)(k < NL ? k : 0) * ncols) + q0;
#pragma unroll
      for (int m = 0; m < NQL; ++m) {
        const int qq = l4 + 4 * m;
        if (q0 + qq < nq) {
          const float4 x = __ldg(Lr + qq);
          acc[m].x = fmaf(t, x.x, acc[m].x);
          acc[m].y = fmaf(t, x.y, acc[m].y);
          acc[m].z = fmaf(t, x.z, acc[m].z);
          acc[m].w = fmaf(t, x.w, acc[m].w);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < NQL; ++m) {
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) {
        acc[m].x += __shfl_xor_sync(0xffffffffu, acc[m].x, o);
        acc[m].y += __shfl_xor_sync(0xffffffffu, acc[m].y, o);
        acc[m].z += __shfl_xor_sync(0xffffffffu, acc[m].z, o);
        acc[m].w += __shfl_xor_sync(0xffffffffu, acc[m].w, o);
      }
    }
    if (g == 0) {
#pragma unroll
      for (int m = 0; m < NQL; ++m) {
        const int qq = l4 + 4 * m;
        if (q0 + qq < nq)
          reinterpret_cast<float4*>(R + (long long)warp * ncols)[q0 + qq] = acc[m];
      }
    }
  }
}

// ---------------------------------------------------------------- bin-CSR FP16
// One warp per (vertex, s), s fastest, so the bin rows of one vertex are reused
// across its shifts from L1.  Lanes take interleaved entries (lane + 32 i):
// the row is sorted by coefficient index, so each warp-wide gather touches
// neighbouring lighting rows L[s][k][c] (channels interleaved), NL
// coefficients per (s, c).
template <bool VEC4>
__global__ void __launch_bounds__(256) k_shade_bincsr_f16(const __half* __restrict__ vals,
                                                          const uint32_t* __restrict__ idx,
                                                          const uint8_t* __restrict__ bin_of, int V,
                                                          int bins, int K, int S, int C,
                                                          const float* __restrict__ L, long long NL,
                                                          float* __restrict__ R) {
  pdl_wait();                                     // inputs come from the previous kernel
  // CTA = 8 vertices x one shift, the shift fastest across CTAs: a CTA's
  // gathers all fall in one shift's lighting plane (L1-resident), and the S
  // CTAs of a vertex block run together, so each stored row they share is
  // fetched from DRAM once
  const int lane = threadIdx.x & 31;
  const long long cta = blockIdx.x;
  const int s = (int)(cta % S);
  const int v = (int)(cta / S) * 8 + (threadIdx.x >> 5);
  if (v >= V) return;
  const int b = __ldg(bin_of + (long long)s * V + v);
  const long long row = ((long long)v * bins + b) * K;
  const int cs = VEC4 ? 4 : C;                              // floats per coefficient
  const float* Ls = L + (long long)s * NL * cs;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int j = lane; j < K; j += 32) {
    const long long k0 = __ldg(idx + row + j);
    const bool ok = k0 < NL;                                // out-of-range entries are ignored
    const float t = ok ? __half2float(vals[row + j]) : 0.0f;
    const float* lk = Ls + (ok ? k0 : 0) * cs;
    if (VEC4) {
      // one 16-byte gather per entry; the pad channel is never accumulated
      const float4 x = __ldg(reinterpret_cast<const float4*>(lk));
      acc[0] = fmaf(t, x.x, acc[0]);
      acc[1] = fmaf(t, x.y, acc[1]);
      acc[2] = fmaf(t, x.z, acc[2]);
      acc[3] = fmaf(t, x.w, acc[3]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (c < C) acc[c] = fmaf(t, __ldg(lk + c), acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float x = acc[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    acc[c] = x;
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < C) R[((long long)v * S + s) * C + c] = acc[c];
  }
}

// ---------------------------------------------------------------- vertex-group CSR
// The top-K sets of neighbouring vertices overlap heavily (4 consecutive
// torus vertices of the 50 000-vertex top-256 scene: ~295 distinct
// coefficients of 4 x 256), so groups of 4 vertices share one sorted union
// index list with values [nnz_g][4] (zero where a vertex lacks the
// coefficient): every lighting row gathered feeds 4 vertices.  (Larger
// groups cut the row gathers further but lose the L1 reuse of the coarse
// rows that every group repeats; 4 measured best.)
constexpr int kGroup = HAAR_GCSR_GROUP;
static_assert(kGroup == 4, "lane layout below assumes 4-vertex groups");

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void l2_prefetch_bulk(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 16 bytes that are used once: past L1, so that L1 keeps the lighting rows
__device__ __forceinline__ float4 ld_stream_f4(const float4* p) {
  float4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

// CTA = 4 groups x 2 warps (a pair per group; the two warps split the
// group's union list in halves and add through shared memory, a named
// barrier per pair).  A warp takes 8 entries per step: lane
// = 4 e + cq, entry slot e, float4 columns cq, cq + 4, ... (NQ of the
// lighting row), and accumulates its columns for the 4 vertices with paired FMAs;
// the 8 slots are summed with shuffles at the end.  The union list streams
// in batches of 32 (indices kept in a register, values staged in shared
// memory), the next batch requested while the current one is used, the
// lighting row of step p + 1 in flight while step p's products issue, and
// the whole half-list sent towards L2 by one bulk prefetch when the group
// starts; the values are read past L1 (no-allocate), which keeps L1 for the
// lighting rows.  Entries past the list's end or with an index >= NL become
// (row 0, value 0), so the inner loop carries no predicate.  EXACT: the row
// is exactly 4 NQ float4 wide (one column pass, no column guards).
template <int NQ, bool EXACT>
__global__ void __launch_bounds__(256, 2) k_shade_gcsr_f32(const float* __restrict__ vals,
                                                           const uint16_t* __restrict__ idx,
                                                           const int32_t* __restrict__ gptr, int V,
                                                           const float* __restrict__ L, int NL, int ncols,
                                                           float* __restrict__ R) {
  pdl_wait();                                     // inputs come from the previous kernel
  typedef unsigned long long u64;
  __shared__ ulonglong2 red[4][4][kGroup][NQ];
  __shared__ float4 sv[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gl = w >> 1, wh = w & 1;
  const int n_groups = (V + kGroup - 1) / kGroup;
  const int es = lane >> 2, cq = lane & 3;
  const int nq = EXACT ? 4 * NQ : (ncols >> 2);
  const float4* V4 = reinterpret_cast<const float4*>(vals);
  const int g = blockIdx.x * 4 + gl;
  if (g < n_groups) {
    const int beg = __ldg(gptr + g), end = __ldg(gptr + g + 1);
    const int mid = beg + (end - beg + 1) / 2;
    const int jb = wh ? mid : beg;
    const int je = wh ? end : mid;
    if (lane == 0 && je > jb) {
      l2_prefetch_bulk(vals + 4ll * jb, 16u * (unsigned)(je - jb));
      const uintptr_t ib = reinterpret_cast<uintptr_t>(idx + jb) & ~uintptr_t(15);
      const uintptr_t ie = reinterpret_cast<uintptr_t>(idx + je) & ~uintptr_t(15);
      if (ie > ib) l2_prefetch_bulk(reinterpret_cast<const void*>(ib), (unsigned)(ie - ib));
    }
    for (int q0 = 0; q0 < nq; q0 += 4 * NQ) {
      // lane cq takes float4 columns q0 + cq + 4 m: each load instruction then
      // reads 64 contiguous bytes of a row (2 sectors), a row costs its 6
      // sectors once; columns beyond the row (generic widths only) read row
      // 0's first float4 and are not stored
      int qoff[NQ];
#pragma unroll
      for (int m = 0; m < NQ; ++m) qoff[m] = (EXACT || q0 + cq + 4 * m < nq) ? q0 + cq + 4 * m : 0;
      u64 acc[kGroup][NQ][2];
#pragma unroll
      for (int v = 0; v < kGroup; ++v)
#pragma unroll
        for (int m = 0; m < NQ; ++m) acc[v][m][0] = acc[v][m][1] = 0ull;
      int nk = 0;
      float4 nv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (jb + lane < je) {
        nk = __ldg(idx + jb + lane);
        nv = ld_stream_f4(V4 + jb + lane);
        if (nk >= NL) { nk = 0; nv = make_float4(0.f, 0.f, 0.f, 0.f); }
      }
      for (int j0 = jb; j0 < je; j0 += 32) {
        const int myk = nk;
        __syncwarp();
        sv[w][lane] = nv;
        __syncwarp();
        const int jn = j0 + 32 + lane;
        nk = 0;
        nv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jn < je) {
          nk = __ldg(idx + jn);
          nv = ld_stream_f4(V4 + jn);
          if (nk >= NL) { nk = 0; nv = make_float4(0.f, 0.f, 0.f, 0.f); }
        }
        const int steps = min(4, (je - j0 + 7) >> 3);           // warp-uniform
        // software pipeline: the lighting row of step p + 1 is in flight while
        // step p's products issue
        ulonglong2 x[NQ];
        {
          const int k = __shfl_sync(0xffffffffu, myk, es);
          const ulonglong2* row = reinterpret_cast<const ulonglong2*>(L) + (unsigned)k * (unsigned)nq;
#pragma unroll
          for (int m = 0; m < NQ; ++m) x[m] = __ldg(row + qoff[m]);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (p < steps) {
            ulonglong2 xn[NQ];
            if (p + 1 < steps) {
              const int k = __shfl_sync(0xffffffffu, myk, 8 * (p + 1) + es);
              const ulonglong2* row = reinterpret_cast<const ulonglong2*>(L) + (unsigned)k * (unsigned)nq;
#pragma unroll
              for (int m = 0; m < NQ; ++m) xn[m] = __ldg(row + qoff[m]);
            }
            const float4 t = sv[w][8 * p + es];
            const u64 tt[4] = {f2_dup(t.x), f2_dup(t.y), f2_dup(t.z), f2_dup(t.w)};
#pragma unroll
            for (int v = 0; v < kGroup; ++v)
#pragma unroll
              for (int m = 0; m < NQ; ++m) {
                acc[v][m][0] = f2_fma(tt[v], x[m].x, acc[v][m][0]);
                acc[v][m][1] = f2_fma(tt[v], x[m].y, acc[v][m][1]);
              }
            if (p + 1 < steps) {
#pragma unroll
              for (int m = 0; m < NQ; ++m) x[m] = xn[m];
            }
          }
        }
      }
      // sum the 8 entry slots (lanes cq, cq + 4, ..., cq + 28)
#pragma unroll
      for (int v = 0; v < kGroup; ++v)
#pragma unroll
        for (int m = 0; m < NQ; ++m)
#pragma unroll
          for (int o = 4; o < 32; o <<= 1) {
            acc[v][m][0] = f2_add(acc[v][m][0], f2_shfl_xor(acc[v][m][0], o));
            acc[v][m][1] = f2_add(acc[v][m][1], f2_shfl_xor(acc[v][m][1], o));
          }
      if (wh == 1 && es == 0) {
#pragma unroll
        for (int v = 0; v < kGroup; ++v)
#pragma unroll
          for (int m = 0; m < NQ; ++m) red[gl][cq][v][m] = make_ulonglong2(acc[v][m][0], acc[v][m][1]);
      }
      pair_sync(1 + gl);
      if (wh == 0 && es == 0) {
#pragma unroll
        for (int v = 0; v < kGroup; ++v) {
          const int vv = g * kGroup + v;
          if (vv < V) {
#pragma unroll
            for (int m = 0; m < NQ; ++m) {
              if (EXACT || q0 + cq + 4 * m < nq) {
                const ulonglong2 o = red[gl][cq][v][m];
                const u64 s0 = f2_add(acc[v][m][0], o.x), s1 = f2_add(acc[v][m][1], o.y);
                reinterpret_cast<ulonglong2*>(R + (long long)vv * ncols)[q0 + cq + 4 * m] = make_ulonglong2(s0, s1);
              }
            }
          }
        }
      }
      pair_sync(1 + gl);
    }
  }
}


// One batch of 4 N entries of the union list (N warp steps, no per-step
// predicates: entries past the list's end are (row 0, value 0)), the rows
// of step p + D requested while step p's products issue.  sw = the warp's
// staged values, myk = lane j's index of entry j of the batch.
template <int N, int D>
__device__ __forceinline__ void gcsr48_batch(unsigned long long (&acc)[kGroup][3], const float4* sw, int myk,
                                             const ulonglong2* La, const unsigned long long* Lb, int es) {
  typedef unsigned long long u64;
  ulonglong2 xa[N];
  u64 xb[N];
#pragma unroll
  for (int p = 0; p < D && p < N; ++p) {
    const int k = __shfl_sync(0xffffffffu, myk, 4 * p + es);
    xa[p] = __ldg(La + (unsigned)k * 12u);
    xb[p] = __ldg(Lb + (unsigned)k * 24u);
  }
#pragma unroll
  for (int p = 0; p < N; ++p) {
    if (p + D < N) {
      const int k = __shfl_sync(0xffffffffu, myk, 4 * (p + D) + es);
      xa[p + D] = __ldg(La + (unsigned)k * 12u);
      xb[p + D] = __ldg(Lb + (unsigned)k * 24u);
    }
    const float4 t = sw[4 * p + es];
    const u64 tt[4] = {f2_dup(t.x), f2_dup(t.y), f2_dup(t.z), f2_dup(t.w)};
#pragma unroll
    for (int v = 0; v < kGroup; ++v) {
      acc[v][0] = f2_fma(tt[v], xa[p].x, acc[v][0]);
      acc[v][1] = f2_fma(tt[v], xa[p].y, acc[v][1]);
      acc[v][2] = f2_fma(tt[v], xb[p], acc[v][2]);
    }
  }
}

// Group-CSR shading for rows of exactly 48 floats (16 shifts x RGB, the c1
// frame): the same CTA = 4 groups x 2 warps and batch staging as
// k_shade_gcsr_f32, but a row is spread over 8 lanes (lane = 8 e + c: entry
// slot e of 4, floats 4c..4c+3 and 32+2c..33+2c of the row), so a lane holds
// 12 paired accumulators (4 vertices x 6 floats) instead of 24.  Each batch of
// 32 entries runs as 8 (or, for the last 16 or fewer, 4) predicate-free warp
// steps with the rows of step p + 3 in flight while step p's products issue
// (80 registers, 3 CTAs per SM).
constexpr int kGcsr48Ahead = 3;

__global__ void __launch_bounds__(256, 3) k_shade_gcsr48(const float* __restrict__ vals,
                                                           const uint16_t* __restrict__ idx,
                                                           const int32_t* __restrict__ gptr, int V,
                                                           const float* __restrict__ L, int NL,
                                                           float* __restrict__ R) {
  // Only the lighting L comes from the previous kernel (the phase shift,
  // launched as this kernel's programmatic primary).  The transport is read
  // before waiting for it: the library's kernels that let dependents start
  // early are the shift kernels, which do not write transport, and every
  // frame's set-up is an ordinary launch (a full stream barrier).  So the
  // first CTAs fetch their entry lists while the shift finishes.
  typedef unsigned long long u64;
  __shared__ u64 red[4][8][kGroup][3];
  __shared__ float4 sv[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gl = w >> 1, wh = w & 1;
  const int n_groups = (V + kGroup - 1) / kGroup;
  const int es = lane >> 3, c8 = lane & 7;
  const float4* V4 = reinterpret_cast<const float4*>(vals);
  const ulonglong2* La = reinterpret_cast<const ulonglong2*>(L) + c8;
  const u64* Lb = reinterpret_cast<const u64*>(L + 32) + c8;
  const int g = blockIdx.x * 4 + gl;
  if (g >= n_groups) return;                      // both warps of a pair leave together
  const int beg = __ldg(gptr + g), end = __ldg(gptr + g + 1);
  const int mid = beg + (end - beg + 1) / 2;
  const int jb = wh ? mid : beg;
  const int je = wh ? end : mid;
  if (lane == 0 && je > jb) {
    l2_prefetch_bulk(vals + 4ll * jb, 16u * (unsigned)(je - jb));
    const uintptr_t ib = reinterpret_cast<uintptr_t>(idx + jb) & ~uintptr_t(15);
    const uintptr_t ie = reinterpret_cast<uintptr_t>(idx + je) & ~uintptr_t(15);
    if (ie > ib) l2_prefetch_bulk(reinterpret_cast<const void*>(ib), (unsigned)(ie - ib));
  }
  u64 acc[kGroup][3];
#pragma unroll
  for (int v = 0; v < kGroup; ++v) acc[v][0] = acc[v][1] = acc[v][2] = 0ull;
  int nk = 0;
  float4 nv = make_float4(0.f, 0.f, 0.f, 0.f);
  if (jb + lane < je) {
    nk = __ldg(idx + jb + lane);
    nv = ld_stream_f4(V4 + jb + lane);
    if (nk >= NL) { nk = 0; nv = make_float4(0.f, 0.f, 0.f, 0.f); }
  }
  pdl_wait();                                     // the lighting is complete
  for (int j0 = jb; j0 < je; j0 += 32) {
    const int myk = nk;
    __syncwarp();
    sv[w][lane] = nv;
    __syncwarp();
    const int jn = j0 + 32 + lane;
    nk = 0;
    nv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (jn < je) {
      nk = __ldg(idx + jn);
      nv = ld_stream_f4(V4 + jn);
      if (nk >= NL) { nk = 0; nv = make_float4(0.f, 0.f, 0.f, 0.f); }
    }
    if (je - j0 > 16) gcsr48_batch<8, kGcsr48Ahead>(acc, sv[w], myk, La, Lb, es);
    else gcsr48_batch<4, kGcsr48Ahead>(acc, sv[w], myk, La, Lb, es);
  }
  // sum the 4 entry slots (lanes c8, c8 + 8, c8 + 16, c8 + 24), then the pair's halves
#pragma unroll
  for (int v = 0; v < kGroup; ++v)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      acc[v][m] = f2_add(acc[v][m], f2_shfl_xor(acc[v][m], 8));
      acc[v][m] = f2_add(acc[v][m], f2_shfl_xor(acc[v][m], 16));
    }
  if (wh == 1 && es == 0) {
#pragma unroll
    for (int v = 0; v < kGroup; ++v)
#pragma unroll
      for (int m = 0; m < 3; ++m) red[gl][c8][v][m] = acc[v][m];
  }
  pair_sync(1 + gl);
  if (wh == 0 && es == 0) {
#pragma unroll
    for (int v = 0; v < kGroup; ++v) {
      const int vv = g * kGroup + v;
      if (vv < V) {
        float* o = R + (long long)vv * 48;
        reinterpret_cast<ulonglong2*>(o)[c8] =
            make_ulonglong2(f2_add(acc[v][0], red[gl][c8][v][0]), f2_add(acc[v][1], red[gl][c8][v][1]));
        reinterpret_cast<u64*>(o + 32)[c8] = f2_add(acc[v][2], red[gl][c8][v][2]);
      }
    }
  }
}

// Packing CSR -> vertex-group CSR.  One warp per group builds the bitmap of
// the union of its rows' indices in shared memory (N <= 65536: 2048 words).
constexpr int kBmWords = 2048;

__device__ void gcsr_bitmap(uint32_t* bm, const int32_t* rowptr, const uint16_t* idx, int V, int N, int g, int lane) {
  for (int w = lane; w < kBmWords; w += 32) bm[w] = 0u;
  __syncwarp();
  for (int vl = 0; vl < kGroup; ++vl) {
    const int v = g * kGroup + vl;
    if (v >= V) break;
    for (int j = rowptr[v] + lane; j < rowptr[v + 1]; j += 32) {
      const int k = idx[j];
      if (k < N) atomicOr(bm + (k >> 5), 1u << (k & 31));
    }
  }
  __syncwarp();
}

__global__ void __launch_bounds__(128) k_gcsr_count(const int32_t* __restrict__ rowptr, const uint16_t* __restrict__ idx,
                                                    int V, int N, int32_t* __restrict__ counts) {
  __shared__ uint32_t bm_all[4][kBmWords];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * 4 + w;
  const int n_groups = (V + kGroup - 1) / kGroup;
  if (g >= n_groups) return;
  uint32_t* bm = bm_all[w];
  gcsr_bitmap(bm, rowptr, idx, V, N, g, lane);
  int c = 0;
  for (int i = lane; i < kBmWords; i += 32) c += __popc(bm[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) counts[g] = c;
}

// exclusive scan of counts[n] into gptr[n + 1] (one block)
__global__ void __launch_bounds__(1024) k_scan(const int32_t* __restrict__ counts, int n, int32_t* __restrict__ gptr) {
  __shared__ int32_t part[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int x = i < n ? counts[i] : 0;
    part[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int y = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < n) gptr[i] = carry + part[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) gptr[n] = carry;
}

__global__ void __launch_bounds__(64) k_gcsr_fill(const int32_t* __restrict__ rowptr, const uint16_t* __restrict__ idx,
                                                  const float* __restrict__ vals, int V, int N,
                                                  const int32_t* __restrict__ gptr, uint16_t* __restrict__ gidx,
                                                  float* __restrict__ gvals) {
  __shared__ uint32_t bm_all[2][kBmWords];
  __shared__ int32_t pre_all[2][kBmWords];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * 2 + w;
  const int n_groups = (V + kGroup - 1) / kGroup;
  if (g >= n_groups) return;
  uint32_t* bm = bm_all[w];
  int32_t* pre = pre_all[w];
  gcsr_bitmap(bm, rowptr, idx, V, N, g, lane);
  // exclusive prefix popcount per word: lane owns 64 consecutive words
  constexpr int per = kBmWords / 32;
  int local = 0;
  for (int i = 0; i < per; ++i) local += __popc(bm[lane * per + i]);
  int incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  int run = incl - local;
  for (int i = 0; i < per; ++i) {
    pre[lane * per + i] = run;
    run += __popc(bm[lane * per + i]);
  }
  __syncwarp();
  const long long base = gptr[g];
  const int cnt = gptr[g + 1] - gptr[g];
  for (int i = 0; i < per; ++i) {
    const int wd = lane * per + i;
    uint32_t bits = bm[wd];
    int p = pre[wd];
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      gidx[base + p] = (uint16_t)(wd * 32 + b);
      ++p;
    }
  }
  for (long long e = lane; e < (long long)cnt * kGroup; e += 32) gvals[base * kGroup + e] = 0.0f;
  __syncwarp();
  for (int vl = 0; vl < kGroup; ++vl) {
    const int v = g * kGroup + vl;
    if (v >= V) break;
    for (int j = rowptr[v] + lane; j < rowptr[v + 1]; j += 32) {
      const int k = idx[j];
      if (k >= N) continue;
      const uint32_t word = bm[k >> 5];
      const int pos = pre[k >> 5] + __popc(word & ((1u << (k & 31)) - 1u));
      gvals[(base + pos) * kGroup + vl] = vals[j];
    }
  }
}

// ---------------------------------------------------------------- view bins
__global__ void k_view_bins(int V, int S, int bins, const float* __restrict__ pos,
                            const float* __restrict__ nrm, const float* __restrict__ cams,
                            const float* __restrict__ bin_dirs, uint8_t* __restrict__ bin_of) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)V * S) return;
  const int s = (int)(e / V), v = (int)(e - (long long)s * V);
  const float nx = nrm[3 * v], ny = nrm[3 * v + 1], nz = nrm[3 * v + 2];
  // branchless orthonormal basis around n (Duff et al. 2017)
  const float sg = nz >= 0.0f ? 1.0f : -1.0f;
  const float a = -1.0f / (sg + nz);
  const float bb = nx * ny * a;
  const float b1x = 1.0f + sg * nx * nx * a, b1y = sg * bb, b1z = -sg * nx;
  const float b2x = bb, b2y = sg + ny * ny * a, b2z = -ny;
  float wx = cams[3 * s] - pos[3 * v], wy = cams[3 * s + 1] - pos[3 * v + 1],
        wz = cams[3 * s + 2] - pos[3 * v + 2];
  const float inv = rsqrtf(wx * wx + wy * wy + wz * wz);
  wx *= inv; wy *= inv; wz *= inv;
  const float lx = wx * b1x + wy * b1y + wz * b1z;
  const float ly = wx * b2x + wy * b2y + wz * b2z;
  const float lz = wx * nx + wy * ny + wz * nz;
  int best = 0;
  float bd = -3.0f;
  for (int b = 0; b < bins; ++b) {
    const float d = lx * bin_dirs[3 * b] + ly * bin_dirs[3 * b + 1] + lz * bin_dirs[3 * b + 2];
    if (d > bd) { bd = d; best = b; }
  }
  bin_of[e] = (uint8_t)best;
}

// ---------------------------------------------------------------- launchers
haar_status_t launch_shade_dense_f32(const float* T, int V, int K, const float* L, int ldl, int ncols,
                                     float* R, cudaStream_t st) {
  const long long threads = (long long)V * 32;
  return cuda_check(launch_pdl(k_shade_dense_f32, dim3((unsigned)((threads + 255) / 256)), dim3(256), 0, st, T, V, K, L, ldl, ncols, R), "k_shade_dense_f32 launch");
}

haar_status_t launch_shade_csr_f32(const float* vals, const uint16_t* idx, const int32_t* rowptr, int V,
                                   const float* L, int NL, int ncols, float* R, cudaStream_t st) {
  const long long threads = (long long)V * 32;
  const unsigned nb = (unsigned)((threads + 255) / 256);
  const int nq = ncols / 4;
  cudaError_t e;
  if (nq <= 4) e = launch_pdl(k_shade_csr_f32<1>, dim3(nb), dim3(256), 0, st, vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 8) e = launch_pdl(k_shade_csr_f32<2>, dim3(nb), dim3(256), 0, st, vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 12) e = launch_pdl(k_shade_csr_f32<3>, dim3(nb), dim3(256), 0, st, vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 16) e = launch_pdl(k_shade_csr_f32<4>, dim3(nb), dim3(256), 0, st, vals, idx, rowptr, V, L, NL, ncols, R);
  else e = launch_pdl(k_shade_csr_f32<8>, dim3(nb), dim3(256), 0, st, vals, idx, rowptr, V, L, NL, ncols, R);
  return cuda_check(e, "k_shade_csr_f32 launch");
}

haar_status_t launch_shade_gcsr_f32(const float* vals, const uint16_t* idx, const int32_t* gptr, int V,
                                    const float* L, int NL, int ncols, float* R, int* status, cudaStream_t st) {
  (void)status;
  const int nq = ncols / 4;
  const long long groups = (V + kGroup - 1) / kGroup;
  const unsigned nb = (unsigned)((groups + 3) / 4);
  cudaError_t e;
  if (nq == 12) e = launch_pdl(k_shade_gcsr48, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, R);
  else if (nq == 8) e = launch_pdl(k_shade_gcsr_f32<2, true>, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, ncols, R);
  else if (nq == 4) e = launch_pdl(k_shade_gcsr_f32<1, true>, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, ncols, R);
  else if (nq <= 4) e = launch_pdl(k_shade_gcsr_f32<1, false>, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, ncols, R);
  else if (nq <= 8) e = launch_pdl(k_shade_gcsr_f32<2, false>, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, ncols, R);
  else e = launch_pdl(k_shade_gcsr_f32<3, false>, dim3(nb), dim3(256), 0, st, vals, idx, gptr, V, L, NL, ncols, R);   // 48-column passes
  return cuda_check(e, "k_shade_gcsr_f32 launch");
}

haar_status_t launch_gcsr_pack(int V, int N, const int32_t* rowptr, const uint16_t* idx, const float* vals,
                               int32_t* gptr, uint16_t* gidx, float* gvals, cudaStream_t st) {
  const int groups = (V + kGroup - 1) / kGroup;
  // counts go to gptr[1..groups] first, then the scan turns them into offsets in place
  int32_t* counts = gptr + 1;
  k_gcsr_count<<<(groups + 3) / 4, 128, 0, st>>>(rowptr, idx, V, N, counts);
  haar_status_t r = cuda_check(cudaGetLastError(), "k_gcsr_count launch");
  if (r != HAAR_OK) return r;
  k_scan<<<1, 1024, 0, st>>>(counts, groups, gptr);
  r = cuda_check(cudaGetLastError(), "k_scan launch");
  if (r != HAAR_OK || gidx == nullptr) return r;
  k_gcsr_fill<<<(groups + 1) / 2, 64, 0, st>>>(rowptr, idx, vals, V, N, gptr, gidx, gvals);
  return cuda_check(cudaGetLastError(), "k_gcsr_fill launch");
}

haar_status_t launch_shade_bincsr_f16(const __half* vals, const uint32_t* idx, const uint8_t* bin_of,
                                      int V, int bins, int K, int S, int C, const float* L, long long NL,
                                      bool vec4, float* R, cudaStream_t st) {
  const dim3 grid((unsigned)(((long long)V + 7) / 8 * S));
  const cudaError_t e =
      vec4 ? launch_pdl(k_shade_bincsr_f16<true>, grid, dim3(256), 0, st, vals, idx, bin_of, V, bins, K, S, C, L, NL, R)
           : launch_pdl(k_shade_bincsr_f16<false>, grid, dim3(256), 0, st, vals, idx, bin_of, V, bins, K, S, C, L, NL, R);
  return cuda_check(e, "k_shade_bincsr_f16 launch");
}

haar_status_t launch_view_bins(int V, int S, int bins, const float* pos, const float* nrm,
                               const float* cams, const float* bin_dirs, uint8_t* bin_of,
                               cudaStream_t st) {
  const long long n = (long long)V * S;
  k_view_bins<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, S, bins, pos, nrm, cams, bin_dirs, bin_of);
  return cuda_check(cudaGetLastError(), "k_view_bins launch");
}

}  // namespace hs
