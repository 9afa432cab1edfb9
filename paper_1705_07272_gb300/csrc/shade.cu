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

namespace hs {

// ---------------------------------------------------------------- dense FP32
// One warp per vertex; lanes stride over k with float4 loads; up to 8 output
// columns (s, c) per pass over the row.
__global__ void __launch_bounds__(256) k_shade_dense_f32(const float* __restrict__ T, int V, int K,
                                                         const float* __restrict__ L, int ldl, int ncols,
                                                         float* __restrict__ R) {
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
// One warp per (vertex, s), vertex-major so the bins of one vertex are reused
// across its shifts from L1/L2.  Lighting layout L[s][k][c] (channels
// interleaved), NL coefficients per (s, c).
__global__ void __launch_bounds__(256) k_shade_bincsr_f16(const __half* __restrict__ vals,
                                                          const uint32_t* __restrict__ idx,
                                                          const uint8_t* __restrict__ bin_of, int V,
                                                          int bins, int K, int S, int C,
                                                          const float* __restrict__ L, long long NL,
                                                          float* __restrict__ R) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)V * S) return;
  const int v = (int)(warp / S), s = (int)(warp - (long long)v * S);
  const int b = __ldg(bin_of + (long long)s * V + v);
  const long long row = ((long long)v * bins + b) * K;
  const float* Ls = L + (long long)s * NL * C;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int j = lane; j < K; j += 32) {
    const long long k0 = __ldg(idx + row + j);
    const bool ok = k0 < NL;                                // out-of-range entries are ignored
    const float t = ok ? __half2float(vals[row + j]) : 0.0f;
    const float* lk = Ls + (ok ? k0 : 0) * C;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < C) acc[c] = fmaf(t, __ldg(lk + c), acc[c]);
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
  k_shade_dense_f32<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(T, V, K, L, ldl, ncols, R);
  return cuda_check(cudaGetLastError(), "k_shade_dense_f32 launch");
}

haar_status_t launch_shade_csr_f32(const float* vals, const uint16_t* idx, const int32_t* rowptr, int V,
                                   const float* L, int NL, int ncols, float* R, cudaStream_t st) {
  const long long threads = (long long)V * 32;
  const unsigned nb = (unsigned)((threads + 255) / 256);
  const int nq = ncols / 4;
  if (nq <= 4) k_shade_csr_f32<1><<<nb, 256, 0, st>>>(vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 8) k_shade_csr_f32<2><<<nb, 256, 0, st>>>(vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 12) k_shade_csr_f32<3><<<nb, 256, 0, st>>>(vals, idx, rowptr, V, L, NL, ncols, R);
  else if (nq <= 16) k_shade_csr_f32<4><<<nb, 256, 0, st>>>(vals, idx, rowptr, V, L, NL, ncols, R);
  else k_shade_csr_f32<8><<<nb, 256, 0, st>>>(vals, idx, rowptr, V, L, NL, ncols, R);
  return cuda_check(cudaGetLastError(), "k_shade_csr_f32 launch");
}

haar_status_t launch_shade_bincsr_f16(const __half* vals, const uint32_t* idx, const uint8_t* bin_of,
                                      int V, int bins, int K, int S, int C, const float* L, long long NL,
                                      float* R, cudaStream_t st) {
  const long long threads = (long long)V * S * 32;
  k_shade_bincsr_f16<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(vals, idx, bin_of, V, bins, K, S,
                                                                        C, L, NL, R);
  return cuda_check(cudaGetLastError(), "k_shade_bincsr_f16 launch");
}

haar_status_t launch_view_bins(int V, int S, int bins, const float* pos, const float* nrm,
                               const float* cams, const float* bin_dirs, uint8_t* bin_of,
                               cudaStream_t st) {
  const long long n = (long long)V * S;
  k_view_bins<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(V, S, bins, pos, nrm, cams, bin_dirs, bin_of);
  return cuda_check(cudaGetLastError(), "k_view_bins launch");
}

}  // namespace hs
