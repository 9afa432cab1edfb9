// haar_shift_noalloc: the phase shift without a plan and without any
// device allocation.
//
// Some callers cannot allocate device memory: plug-ins inside a host renderer
// or engine whose device memory is owned by the host's own allocator, and
// real-time frame loops that may not call cudaMalloc/cudaFree (they
// synchronise the device and can stall a frame).  This entry point runs the
// same set-up and shift kernels as haar_shift, but its scratch (pixel map,
// sin/cos tables, shift records, tile means, tile counters) lives in one
// file-scope __device__ array of fixed size, so the caller passes only inputs
// and outputs.
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace hs {

// 2 Mi floats = 8 MiB of scratch, held by every GPU that loads the library
// until the process exits.
constexpr size_t kNoAllocFloats = size_t(2) << 20;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
static float* g_noalloc_ptr[kMaxDevices];
static std::mutex g_noalloc_mu;

static size_t round64(size_t x) { return (x + 63) & ~size_t(63); }

}  // namespace hs

using namespace hs;

extern "C" haar_status_t haar_shift_noalloc(const haar_shift_desc_t* d, const float* cin, const double* params,
                                            int S, void* out, void* stream) {
  clear_error();
  if (injected("haar_shift_noalloc")) return set_error(HAAR_ERR_INJECTED, "haar_shift_noalloc: injected fault");
  if (d == nullptr || cin == nullptr || params == nullptr || out == nullptr)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: null argument");
  const int C = d->channels;
  if (d->height < 2 || d->height > 4096 || (d->height & (d->height - 1)) != 0 ||
      (d->width != d->height && d->width != 2 * d->height))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: unsupported map %dx%d", d->height, d->width);
  if (d->start_level < 0 || d->start_level > 12 || (d->height >> d->start_level) < 2)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: start_level %d leaves a map smaller than 2 x 2",
                     d->start_level);
  const int H = d->height >> d->start_level, W = d->width >> d->start_level;   // the map the shift runs on
  if (C < 1 || C > 64) return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: channels %d not in [1, 64]", C);
  if (d->kind == HAAR_SHIFT_ROTATE_CHAIN)
    return set_error(HAAR_ERR_UNSUPPORTED, "haar_shift_noalloc: ROTATE_CHAIN needs a plan (field workspace)");
  if (d->kind < HAAR_SHIFT_TRANSLATE || d->kind > HAAR_SHIFT_ROTATE_EULER ||
      (d->boundary != HAAR_BOUNDARY_SPHERE && d->boundary != HAAR_BOUNDARY_TORUS) ||
      d->out_type < HAAR_OUT_F32 || d->out_type > HAAR_OUT_F16 || d->out_layout < HAAR_LAYOUT_SCK ||
      d->out_layout > HAAR_LAYOUT_SKC4 || (d->out_layout == HAAR_LAYOUT_SKC4 && d->channels > 4))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: unknown kind, boundary, out_type or out_layout");
  const long long N = (long long)H * W;
  if (d->out_coeffs < 0 || d->out_coeffs > N)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: out_coeffs %d not in [0, %lld]", d->out_coeffs, N);
  if (S < 1 || S > 65535) return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: S = %d not in [1, 65535]", S);
  const size_t elem = d->out_type == HAAR_OUT_F32 ? 4 : 2;
  if (((uintptr_t)cin % 4) || ((uintptr_t)params % 8) || ((uintptr_t)out % elem))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_noalloc: misaligned pointer");

  // scratch layout (floats, each region 256-byte aligned)
  const Geometry g = make_geometry(H, W, C, d->boundary, choose_tile(H, W, C, S));
  const bool rot = d->kind == HAAR_SHIFT_ROTATE || d->kind == HAAR_SHIFT_ROTATE_EULER;
  const size_t n_pix = round64((size_t)pix_floats(d->kind, H, W, C));
  const size_t n_trig = round64((size_t)trig_floats(H, W));
  const size_t n_rtab = rot ? round64((size_t)S * 4 * rot_table_float4s(H, W)) : 0;
  const size_t n_prm = round64((size_t)S * sizeof(ShiftParam) / sizeof(float));
  size_t n_means = round64((size_t)S * C * g.n_tiles);
  if (ksc_eligible(*d, g, S) && round64(ksc_means_floats(g, S)) > n_means) n_means = round64(ksc_means_floats(g, S));
  const size_t n_cnt = round64((size_t)S);
  const size_t need = n_pix + n_trig + n_rtab + n_prm + n_means + n_cnt;
  if (need > kNoAllocFloats)
    return set_error(HAAR_ERR_INVALID_ARG,
                     "haar_shift_noalloc: needs %zu scratch floats (pixel map, tables and S = %d shift records), "
                     "the fixed maximum is %zu", need, S, kNoAllocFloats);

  // once per device: the device address of the scratch array (kept for the
  // life of the process; a device reset after the first call is not supported)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "haar_shift_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(HAAR_ERR_UNSUPPORTED, "haar_shift_noalloc: device %d", dev);
  float* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_check(e, "haar_shift_noalloc: cudaGetSymbolAddress");
      g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    base = g_noalloc_ptr[dev];
  }

  haar_shift_plan_s p;
  memset(&p, 0, sizeof(p));
  p.desc = *d;
  p.desc.max_shifts = S;
  p.geo = g;
  p.K = d->out_coeffs ? d->out_coeffs : (int)N;
  p.cin_stride = (long long)d->height * d->width;
  p.pscale = 1.0 / (double)(1 << d->start_level);
  p.device = dev;
  float* q = base;
  p.pix = q;
  q += n_pix;
  p.trig = q;
  q += n_trig;
  p.rtab = rot ? q : nullptr;
  q += n_rtab;
  p.prm = reinterpret_cast<ShiftParam*>(q);
  q += n_prm;
  p.means = q;
  p.means_cap = n_means;
  q += n_means;
  p.counters = reinterpret_cast<unsigned*>(q);
  cudaStream_t st = (cudaStream_t)stream;
  haar_status_t r = HAAR_OK;
  if (d->kind != HAAR_SHIFT_TRANSLATE) r = launch_trig(&p, st);     // tables of this call's map
  if (r == HAAR_OK) r = launch_setup(&p, cin, params, out, S, st);   // also zeroes the tile counters
  if (r == HAAR_OK) r = launch_shift(&p, cin, S, out, st);
  return r;
}
