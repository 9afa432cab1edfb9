// Dense double product on the 5th-generation tensor cores (tcgen05, sm_103a):
//   R[v][j] = sum_k T[v][k] * (Lhi[j][k] + Llo[j][k]),   j = s*C + c,
// with T the per-vertex transport (the lowest K canonical Haar coefficients,
// bfloat16) and L the shifted lighting split into bfloat16 hi + lo parts, so
// the product keeps ~16 mantissa bits of the lighting while the transport
// streams from HBM as bfloat16 (Eq. 2-5 with two factors, Parseval).
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0     TMA producer: A tile [128 x 64] of T and the B tiles [N x 64]
//              of Lhi and Llo per k-block into a 3-stage ring (128-byte swizzle),
//              the A tile kPrefetchA k-blocks ahead sent towards L2 first;
//   warp 1     TMEM allocator and MMA issuer: for every k-block 4 x 2
//              tcgen05.mma (M=128, N, K=16) accumulate T*Lhi + T*Llo into an
//              FP32 accumulator in tensor memory (two accumulators, so the
//              epilogue of one vertex tile overlaps the next tile's MMAs);
//   warps 2-5  epilogue: tcgen05.ld the accumulator rows and store them.
// Every mbarrier wait is bounded (by %globaltimer); on expiry the kernel
// records HAAR_ERR_TIMEOUT in the status word, drains what it issued, frees
// its tensor memory and returns.
#include "tc.cuh"

namespace hs {
namespace tc {

constexpr int THREADS = 192;       // 6 warps
// k-blocks of transport prefetched into L2 ahead of the ring (measured on the
// 200 000 x 4096 x 192 contraction: 0 -> 0.493 ms, 4 -> 0.463, 8 -> 0.463,
// 16 -> 0.477, 32 -> 0.590)
constexpr int kPrefetchA = 4;

struct __align__(8) Bars {
  uint64_t full[MAX_STAGES];
  uint64_t empty[MAX_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

// A CTA's work: `rounds` whole vertex tiles (blockIdx.x + i gridDim.x), then,
// when the tiles do not divide evenly over the CTAs, its part of one of the
// remaining tiles, each split into tail_p column slices of N / tail_p (so the
// last round costs 1 / tail_p of a tile instead of one whole tile on a few
// CTAs).  part < 0: all N columns.
struct DenseWork {
  int tile, part;
};
__device__ __forceinline__ bool dense_work(int i, int n_tiles, int rounds, int tail_p, DenseWork& w) {
  if (tail_p <= 1) {
    w.tile = blockIdx.x + i * gridDim.x;
    w.part = -1;
    return w.tile < n_tiles;
  }
  if (i < rounds) {
    w.tile = blockIdx.x + i * gridDim.x;
    w.part = -1;
    return true;
  }
  if (i == rounds && (int)blockIdx.x < (n_tiles - rounds * (int)gridDim.x) * tail_p) {
    w.tile = rounds * gridDim.x + blockIdx.x / tail_p;
    w.part = blockIdx.x % tail_p;
    return true;
  }
  return false;
}

__global__ void __launch_bounds__(THREADS, 1)
k_dense_bf16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBh,
             const __grid_constant__ CUtensorMap mapBl, const __grid_constant__ CUtensorMap mapBhT,
             const __grid_constant__ CUtensorMap mapBlT, int V, int K, int N, int STAGES, int tail_p,
             float* __restrict__ R, int* status, int pf_dist) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ Bars bars;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // 1024-byte aligned ring: per stage A (16 KB) | Bhi (N*128 B) | Blo (N*128 B)
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)N * BK * 2;
  const uint32_t stage_bytes = a_bytes + 2 * b_bytes;
  const int n_tiles = (V + BM - 1) / BM;
  const int rounds = n_tiles / (int)gridDim.x;
  const int NT = N / (tail_p > 1 ? tail_p : 1);           // columns of a tail slice
  const uint32_t bt_bytes = (uint32_t)NT * BK * 2;
  const int kblocks = K / BK;
  volatile int* abort_flag = &bars.abort_flag;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&bars.full[s]), 1);
      mbar_init(smem_u32(&bars.empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&bars.tfull[a]), 1);
      mbar_init(smem_u32(&bars.tempty[a]), 4);
    }
    mbar_init(smem_u32(&bars.drain), 1);
    bars.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {  // whole warp allocates 512 TMEM columns (two N <= 256 accumulators)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&bars.tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = bars.tmem_base;
  pdl_wait();                                     // set-up above overlaps the kernel that wrote the lighting

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapBh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapBl)) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      int issued[MAX_STAGES];
      uint32_t issued_phase[MAX_STAGES];
      for (int i = 0; i < MAX_STAGES; ++i) { issued[i] = 0; issued_phase[i] = 0; }
      bool ok = true;
      // the transport tile of the k-block kPrefetchA blocks ahead heads for L2
      // (it streams from HBM; the lighting tiles stay in L2), so the ring's
      // stages wait on L2 rather than on DRAM latency
      int pf_i = 0, pf_kb = 0;
      DenseWork pw;
      bool pf_on = pf_dist > 0 && dense_work(0, n_tiles, rounds, tail_p, pw);
      auto pf_step = [&]() {
        tma_prefetch_2d(&mapA, pf_kb * BK, pw.tile * BM);
        if (++pf_kb == kblocks) {
          pf_kb = 0;
          pf_on = dense_work(++pf_i, n_tiles, rounds, tail_p, pw);
        }
      };
      for (int i = 0; i < pf_dist && pf_on; ++i) pf_step();
      DenseWork w;
      for (int wi = 0; ok && dense_work(wi, n_tiles, rounds, tail_p, w); ++wi) {
        const bool tail = w.part >= 0;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (pf_on) pf_step();
          if (!mbar_wait(smem_u32(&bars.empty[stage]), phase ^ 1u, status, abort_flag)) { ok = false; break; }
          const uint32_t sa = base + stage * stage_bytes;
          const uint32_t fb = smem_u32(&bars.full[stage]);
          mbar_arrive_tx(fb, a_bytes + 2 * (tail ? bt_bytes : b_bytes));
          tma_load_2d(sa, &mapA, kb * BK, w.tile * BM, fb);
          if (tail) {
            tma_load_2d(sa + a_bytes, &mapBhT, kb * BK, w.part * NT, fb);
            tma_load_2d(sa + a_bytes + b_bytes, &mapBlT, kb * BK, w.part * NT, fb);
          } else {
            tma_load_2d(sa + a_bytes, &mapBh, kb * BK, 0, fb);
            tma_load_2d(sa + a_bytes + b_bytes, &mapBl, kb * BK, 0, fb);
          }
          issued[stage] = 1;
          issued_phase[stage] = phase;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      // every load issued lands before the CTA exits (on the normal path the
      // MMA thread has already consumed them all and these waits pass at once)
      for (int i = 0; i < STAGES; ++i) {
        if (!issued[i]) continue;
        const unsigned long long t0 = gtimer();
        while (!mbar_try(smem_u32(&bars.full[i]), issued_phase[i]) && gtimer() - t0 < TIMEOUT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc_full = make_idesc(BM, N), idesc_tail = make_idesc(BM, NT);
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      bool ok = true;
      DenseWork w;
      for (; ok && dense_work(it, n_tiles, rounds, tail_p, w); ++it) {
        const uint32_t idesc = w.part >= 0 ? idesc_tail : idesc_full;
        const int acc = it & 1;
        const uint32_t accp = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait(smem_u32(&bars.tempty[acc]), accp ^ 1u, status, abort_flag)) { ok = false; break; }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * 256);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(smem_u32(&bars.full[stage]), phase, status, abort_flag)) { ok = false; break; }
          fence_after();
          const uint32_t sa = base + stage * stage_bytes;
#pragma unroll
          for (int k = 0; k < BK / UMMA_K; ++k) {
            const uint64_t da = make_desc(sa + k * UMMA_K * 2);
            const uint64_t dh = make_desc(sa + a_bytes + k * UMMA_K * 2);
            const uint64_t dl = make_desc(sa + a_bytes + b_bytes + k * UMMA_K * 2);
            mma_bf16(d, da, dh, idesc, (kb | k) != 0 ? 1u : 0u);
            mma_bf16(d, da, dl, idesc, 1u);
          }
          mma_commit(smem_u32(&bars.empty[stage]));     // frees the stage when these MMAs finish
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(smem_u32(&bars.tfull[acc]));         // accumulator ready for the epilogue
      }
      // all MMAs issued by this thread complete before tensor memory is freed
      mma_commit(smem_u32(&bars.drain));
      const unsigned long long t0 = gtimer();
      while (!mbar_try(smem_u32(&bars.drain), 0) && gtimer() - t0 < TIMEOUT_NS) {
      }
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter = warp % 4
    const int quarter = warp & 3;
    const int row_in_tile = quarter * 32 + lane;
    int it = 0;
    DenseWork w;
    for (; dense_work(it, n_tiles, rounds, tail_p, w); ++it) {
      const int acc = it & 1;
      const uint32_t accp = (uint32_t)((it >> 1) & 1);
      if (!mbar_wait(smem_u32(&bars.tfull[acc]), accp, status, abort_flag)) break;
      fence_after();
      const long long row = (long long)w.tile * BM + row_in_tile;
      const uint32_t t_row = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * 256);
      const int ncols = w.part >= 0 ? NT : N, col0 = w.part >= 0 ? w.part * NT : 0;
      for (int c0 = 0; c0 < ncols; c0 += 16) {
        float v[16];
        tmem_ld16(t_row + (uint32_t)c0, v);
        if (row < V) {
          float4* dst = reinterpret_cast<float4*>(R + row * N + col0 + c0);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
          dst[2] = make_float4(v[8], v[9], v[10], v[11]);
          dst[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bars.tempty[acc]));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

}  // namespace tc

haar_status_t launch_shade_dense_bf16_tc(const __nv_bfloat16* T, int V, int K, const __nv_bfloat16* Lhi,
                                         const __nv_bfloat16* Llo, int ncols, float* R, int* status,
                                         cudaStream_t st) {
  using namespace tc;
  if (K % BK != 0 || ncols % 16 != 0 || ncols < 16 || ncols > 256)
    return set_error(HAAR_ERR_UNSUPPORTED, "dense bf16 contraction: K %% 64 == 0 and 16 <= S*C <= 256, S*C %% 16 == 0");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the tiles left after whole rounds over the CTAs are split into the most
  // column slices (multiples of 16 columns) that still give each CTA at most one
  const int n_tiles_h = (V + BM - 1) / BM;
  const int grid_h = n_tiles_h < sms ? n_tiles_h : sms;
  const int rem = n_tiles_h % grid_h;
  int tail_p = 1;
  if (rem > 0)
    for (int p = 2; p <= ncols / 16; ++p)
      if (ncols % (16 * p) == 0 && rem * p <= grid_h) tail_p = p;
  CUtensorMap mA, mBh, mBl, mBhT, mBlT;
  const uint32_t nt = (uint32_t)(ncols / tail_p);
  if (!encode_2d(&mA, T, (uint64_t)K, (uint64_t)V, BK, BM) ||
      !encode_2d(&mBh, Lhi, (uint64_t)K, (uint64_t)ncols, BK, (uint32_t)ncols) ||
      !encode_2d(&mBl, Llo, (uint64_t)K, (uint64_t)ncols, BK, (uint32_t)ncols) ||
      !encode_2d(&mBhT, Lhi, (uint64_t)K, (uint64_t)ncols, BK, nt) ||
      !encode_2d(&mBlT, Llo, (uint64_t)K, (uint64_t)ncols, BK, nt))
    return set_error(HAAR_ERR_CUDA, "dense bf16 contraction: cuTensorMapEncodeTiled failed");
  const int n_tiles = (V + BM - 1) / BM;
  const int grid = n_tiles < sms ? n_tiles : sms;
  const size_t stage_bytes = BM * BK * 2 + 2 * (size_t)ncols * BK * 2;
  int stages = (int)(SMEM_BUDGET / stage_bytes);
  if (stages > MAX_STAGES) stages = MAX_STAGES;
  const size_t smem = (size_t)stages * stage_bytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_dense_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(k_dense_bf16)");
  return cuda_check(launch_pdl(k_dense_bf16, dim3(grid), dim3(THREADS), smem, st, mA, mBh, mBl, mBhT, mBlT, V, K,
                              ncols, stages, tail_p, R, status, kPrefetchA),
                    "k_dense_bf16 launch");
}

}  // namespace hs
