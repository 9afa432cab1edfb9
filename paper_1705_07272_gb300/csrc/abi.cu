// C ABI of the Haar phase-shift library: argument validation, plan and
// workspace management, error reporting and dispatch to the kernels.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "common.cuh"

namespace hs {

static thread_local char g_err[512];

haar_status_t set_error(haar_status_t st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { g_err[0] = 0; }

haar_status_t cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HAAR_OK;
  cudaGetLastError();  // a non-sticky failure must not surface again at the next launch
  return set_error(HAAR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// HAAR_FAULT_INJECT: comma-separated entry point names (or "*").
bool injected(const char* entry) {
  const char* s = getenv("HAAR_FAULT_INJECT");
  if (s == nullptr || *s == 0) return false;
  const size_t n = strlen(entry);
  while (*s) {
    const char* e = strchr(s, ',');
    const size_t len = e ? (size_t)(e - s) : strlen(s);
    if ((len == 1 && s[0] == '*') || (len == n && strncmp(s, entry, n) == 0)) return true;
    if (!e) break;
    s = e + 1;
  }
  return false;
}

static bool is_pow2(long long x) { return x > 0 && (x & (x - 1)) == 0; }
static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

static void free_plan(haar_shift_plan_s* p) {
  if (!p) return;
  cudaFree(p->pix);
  cudaFree(p->pixE);
  cudaFree(p->trig);
  cudaFree(p->rtab);
  cudaFree(p->prm);
  cudaFree(p->means);
  cudaFree(p->counters);
  cudaFree(p->light);
  cudaFree(p->status);
  cudaFree(p->chain_ws);
  delete p;
}

static size_t out_elem_bytes(int out_type) { return out_type == HAAR_OUT_F32 ? 4 : 2; }

}  // namespace hs

using namespace hs;

#define HS_ENTRY(name)                                                        \
  g_err[0] = 0;                                                               \
  if (injected(name)) return set_error(HAAR_ERR_INJECTED, "%s: injected fault", name)

extern "C" {

const char* haar_last_error(void) { return g_err; }

const char* haar_version(void) { return "haarshift 0.1 (sm_103a)"; }

haar_status_t haar_shift_plan(const haar_shift_desc_t* d, haar_shift_plan_t* out) {
  HS_ENTRY("haar_shift_plan");
  if (d == nullptr || out == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: null argument");
  *out = nullptr;
  if (!is_pow2(d->height) || d->height < 2 || d->height > 4096)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: height %d is not a power of two in [2, 4096]", d->height);
  if (d->width != d->height && d->width != 2 * d->height)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: width %d must be height or 2*height", d->width);
  if (d->channels < 1 || d->channels > 64)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: channels %d not in [1, 64]", d->channels);
  if (d->kind < HAAR_SHIFT_TRANSLATE || d->kind > HAAR_SHIFT_ROTATE_CHAIN)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: unknown kind %d", d->kind);
  if (d->kind == HAAR_SHIFT_ROTATE_CHAIN && d->out_type != HAAR_OUT_F32)
    return set_error(HAAR_ERR_UNSUPPORTED, "haar_shift_plan: ROTATE_CHAIN writes float32 only");
  if (d->boundary != HAAR_BOUNDARY_SPHERE && d->boundary != HAAR_BOUNDARY_TORUS)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: unknown boundary %d", d->boundary);
  if (d->max_shifts < 1 || d->max_shifts > 65535)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: max_shifts %d not in [1, 65535]", d->max_shifts);
  if (d->start_level < 0 || d->start_level > 12 || (d->height >> d->start_level) < 2)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: start_level %d leaves a map smaller than 2 x 2",
                     d->start_level);
  if (d->kind == HAAR_SHIFT_ROTATE_CHAIN && (d->height >> d->start_level) < 16)
    return set_error(HAAR_ERR_UNSUPPORTED, "haar_shift_plan: ROTATE_CHAIN needs a map of at least 16 rows");
  const int Hk = d->height >> d->start_level, Wk = d->width >> d->start_level;
  const long long N = (long long)Hk * Wk;          // coefficients of the map the shift runs on
  if (d->out_coeffs < 0 || d->out_coeffs > N)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: out_coeffs %d not in [0, %lld]", d->out_coeffs, N);
  if (d->out_type < HAAR_OUT_F32 || d->out_type > HAAR_OUT_F16)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: unknown out_type %d", d->out_type);
  if (d->out_layout < HAAR_LAYOUT_SCK || d->out_layout > HAAR_LAYOUT_SKC4)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: unknown out_layout %d", d->out_layout);
  if (d->out_layout == HAAR_LAYOUT_SKC4 && d->channels > 4)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan: SKC4 holds at most 4 channels (got %d)", d->channels);

  haar_shift_plan_s* p = new (std::nothrow) haar_shift_plan_s();
  if (!p) return set_error(HAAR_ERR_NOMEM, "haar_shift_plan: host allocation failed");
  memset(p, 0, sizeof(*p));
  p->desc = *d;
  p->geo = make_geometry(Hk, Wk, d->channels, d->boundary, choose_tile(Hk, Wk, d->channels, d->max_shifts));
  p->K = d->out_coeffs ? d->out_coeffs : (int)N;
  p->cin_stride = (long long)d->height * d->width;
  p->pscale = 1.0 / (double)(1 << d->start_level);
  cudaGetDevice(&p->device);
  const Geometry& g = p->geo;
  const size_t S = d->max_shifts;
  p->light_elems = S * (d->out_layout == HAAR_LAYOUT_SKC4 ? 4 : g.C) * (size_t)p->K;
  const size_t light_bytes =
      p->light_elems * out_elem_bytes(d->out_type) * (d->out_type == HAAR_OUT_BF16_HILO ? 2 : 1);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&p->pix, sizeof(float) * pix_floats(d->kind, g.H, g.W, g.C));
  if (e == cudaSuccess && tr8_tma_plan(*d, g, p->K, (int)S)) {
    p->pixE_H = ((d->boundary == HAAR_BOUNDARY_SPHERE) ? 2 * g.H : g.H) + 65;
    p->pixE_W = g.W + 68;
    e = cudaMalloc(&p->pixE, sizeof(float) * (size_t)g.C * p->pixE_H * p->pixE_W);
  }
  if (e == cudaSuccess) e = cudaMalloc(&p->trig, sizeof(float) * trig_floats(g.H, g.W));
  if (e == cudaSuccess && (d->kind == HAAR_SHIFT_ROTATE || d->kind == HAAR_SHIFT_ROTATE_EULER))
    e = cudaMalloc(&p->rtab, sizeof(float4) * rot_table_float4s(g.H, g.W) * S);
  if (e == cudaSuccess) e = cudaMalloc(&p->prm, sizeof(ShiftParam) * S);
  p->means_cap = S * g.C * g.n_tiles;
  if (ksc_eligible(*d, g, (int)S) && ksc_means_floats(g, (int)S) > p->means_cap)
    p->means_cap = ksc_means_floats(g, (int)S);
  if (e == cudaSuccess) e = cudaMalloc(&p->means, sizeof(float) * p->means_cap);
  if (e == cudaSuccess) e = cudaMalloc(&p->counters, sizeof(unsigned) * S);
  if (e == cudaSuccess) e = cudaMalloc(&p->light, light_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int) * 4);
  if (e == cudaSuccess && d->kind == HAAR_SHIFT_ROTATE_CHAIN)
    e = cudaMalloc(&p->chain_ws, sizeof(float) * chain_ws_floats(g, (int)S));
  if (e != cudaSuccess) {
    free_plan(p);
    return set_error(HAAR_ERR_NOMEM, "haar_shift_plan: workspace allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemset(p->counters, 0, sizeof(unsigned) * S);
  if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    free_plan(p);
    return cuda_check(e, "haar_shift_plan: cudaMemset");
  }
  haar_status_t r = launch_trig(p, 0);
  if (r == HAAR_OK) r = cuda_check(cudaDeviceSynchronize(), "haar_shift_plan: trig tables");
  if (r != HAAR_OK) {
    free_plan(p);
    return r;
  }
  *out = p;
  return HAAR_OK;
}

haar_status_t haar_shift_plan_destroy(haar_shift_plan_t p) {
  HS_ENTRY("haar_shift_plan_destroy");
  if (p == nullptr) return HAAR_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(p);
  return cuda_check(e, "haar_shift_plan_destroy: synchronise");
}

haar_status_t haar_shift_plan_status(haar_shift_plan_t p, int* status_out, int reset) {
  HS_ENTRY("haar_shift_plan_status");
  if (p == nullptr || status_out == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "haar_shift_plan_status: null argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status_out, p->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(p->status, 0, sizeof(int));
  return cuda_check(e, "haar_shift_plan_status");
}

static haar_status_t check_shift_args(haar_shift_plan_t p, const float* cin, const double* params, int S,
                                      const void* out, const char* who) {
  if (p == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "%s: null plan", who);
  if (cin == nullptr || params == nullptr || out == nullptr)
    return set_error(HAAR_ERR_INVALID_ARG, "%s: null pointer", who);
  if (S < 1 || S > p->desc.max_shifts)
    return set_error(HAAR_ERR_INVALID_ARG, "%s: S = %d not in [1, max_shifts = %d]", who, S, p->desc.max_shifts);
  if (!aligned(cin, 4) || !aligned(params, 8) || !aligned(out, out_elem_bytes(p->desc.out_type)))
    return set_error(HAAR_ERR_INVALID_ARG, "%s: misaligned pointer", who);
  return HAAR_OK;
}

haar_status_t haar_shift(haar_shift_plan_t p, const float* cin, const double* params, int S, void* out,
                         void* stream) {
  HS_ENTRY("haar_shift");
  haar_status_t r = check_shift_args(p, cin, params, S, out, "haar_shift");
  if (r != HAAR_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  r = launch_setup(p, cin, params, out, S, st);
  if (r != HAAR_OK) return r;
  if (p->desc.kind == HAAR_SHIFT_ROTATE_CHAIN) return launch_chain(p, params, S, out, st);
  return launch_shift(p, cin, S, out, st);
}

haar_status_t haar_forward(int H, int W, int batch, const float* maps, float* coeffs, float scale,
                           void* stream) {
  HS_ENTRY("haar_forward");
  if (!is_pow2(H) || H < 2 || H > 4096 || (W != H && W != 2 * H))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_forward: unsupported map %dx%d", H, W);
  if (batch < 0 || batch > 65535) return set_error(HAAR_ERR_INVALID_ARG, "haar_forward: batch %d", batch);
  if (batch == 0) return HAAR_OK;
  if (maps == nullptr || coeffs == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "haar_forward: null pointer");
  if (!aligned(maps, 16) || !aligned(coeffs, 4))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_forward: maps must be 16-byte aligned");
  return launch_forward(H, W, batch, maps, coeffs, scale, (cudaStream_t)stream);
}

haar_status_t haar_inverse(int H, int W, int batch, const float* coeffs, float* maps, void* stream) {
  HS_ENTRY("haar_inverse");
  if (!is_pow2(H) || H < 2 || H > 4096 || (W != H && W != 2 * H))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_inverse: unsupported map %dx%d", H, W);
  if (batch < 0) return set_error(HAAR_ERR_INVALID_ARG, "haar_inverse: batch %d", batch);
  if (batch == 0) return HAAR_OK;
  if (maps == nullptr || coeffs == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "haar_inverse: null pointer");
  return launch_inverse(H, W, batch, coeffs, maps, (cudaStream_t)stream);
}

static haar_status_t shade_impl(haar_shift_plan_t p, const haar_transport_desc_t* t, const void* L, int S,
                                float* R, cudaStream_t st, const char* who) {
  if (p == nullptr || t == nullptr || L == nullptr || R == nullptr)
    return set_error(HAAR_ERR_INVALID_ARG, "%s: null argument", who);
  if (S < 1 || S > p->desc.max_shifts)
    return set_error(HAAR_ERR_INVALID_ARG, "%s: S = %d not in [1, max_shifts]", who, S);
  if (t->V < 0 || t->vals == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "%s: bad transport", who);
  if (t->V == 0) return HAAR_OK;
  const int C = p->geo.C;
  const int ncols = S * C;
  const int ot = p->desc.out_type, lay = p->desc.out_layout;
  switch (t->kind) {
    case HAAR_T_DENSE_F32:
      if (ot != HAAR_OUT_F32 || lay != HAAR_LAYOUT_SCK)
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: DENSE_F32 needs F32 lighting in SCK layout", who);
      if (t->K < 1 || t->K > p->K) return set_error(HAAR_ERR_INVALID_ARG, "%s: K = %d > plan K = %d", who, t->K, p->K);
      if (!aligned(t->vals, 16) || !aligned(L, 16))
        return set_error(HAAR_ERR_INVALID_ARG, "%s: transport and lighting must be 16-byte aligned", who);
      return launch_shade_dense_f32((const float*)t->vals, t->V, t->K, (const float*)L, p->K, ncols, R, st);
    case HAAR_T_DENSE_BF16:
      if (ot != HAAR_OUT_BF16_HILO || lay != HAAR_LAYOUT_SCK)
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: DENSE_BF16 needs BF16_HILO lighting in SCK layout", who);
      if (t->K != p->K || (t->K % 64) != 0)
        return set_error(HAAR_ERR_INVALID_ARG, "%s: DENSE_BF16 needs K == plan K and K %% 64 == 0 (K = %d)", who, t->K);
      if (ncols % 16 != 0 || ncols > 256)
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: DENSE_BF16 needs S*C a multiple of 16, at most 256 (got %d)", who, ncols);
      if (!aligned(t->vals, 16) || !aligned(L, 16) || !aligned(R, 16))
        return set_error(HAAR_ERR_INVALID_ARG, "%s: transport, lighting and radiance must be 16-byte aligned", who);
      return launch_shade_dense_bf16_tc((const __nv_bfloat16*)t->vals, t->V, t->K, (const __nv_bfloat16*)L,
                                        (const __nv_bfloat16*)L + (size_t)S * C * p->K, ncols, R, p->status, st);
    case HAAR_T_CSR_F32_U16:
      if (ot != HAAR_OUT_F32 || lay != HAAR_LAYOUT_KSC)
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: CSR_F32_U16 needs F32 lighting in KSC layout", who);
      if (ncols % 4 != 0) return set_error(HAAR_ERR_UNSUPPORTED, "%s: CSR needs S*C %% 4 == 0", who);
      if (t->idx == nullptr || t->rowptr == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "%s: CSR needs idx and rowptr", who);
      if (!aligned(L, 16) || !aligned(R, 16))
        return set_error(HAAR_ERR_INVALID_ARG, "%s: lighting and radiance must be 16-byte aligned", who);
      if (p->K > 65536) return set_error(HAAR_ERR_UNSUPPORTED, "%s: uint16 indices cover at most 65536 coefficients", who);
      return launch_shade_csr_f32((const float*)t->vals, (const uint16_t*)t->idx, t->rowptr, t->V, (const float*)L,
                                  p->K, ncols, R, st);
    case HAAR_T_GCSR_F32_U16:
      if (ot != HAAR_OUT_F32 || lay != HAAR_LAYOUT_KSC)
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: GCSR_F32_U16 needs F32 lighting in KSC layout", who);
      if (ncols % 4 != 0) return set_error(HAAR_ERR_UNSUPPORTED, "%s: GCSR needs S*C %% 4 == 0", who);
      if (t->idx == nullptr || t->rowptr == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "%s: GCSR needs idx and rowptr", who);
      if (!aligned(L, 16) || !aligned(R, 16) || !aligned(t->vals, 16))
        return set_error(HAAR_ERR_INVALID_ARG, "%s: group values, lighting and radiance must be 16-byte aligned", who);
      if (p->K > 65536) return set_error(HAAR_ERR_UNSUPPORTED, "%s: uint16 indices cover at most 65536 coefficients", who);
      return launch_shade_gcsr_f32((const float*)t->vals, (const uint16_t*)t->idx, t->rowptr, t->V, (const float*)L,
                                   p->K, ncols, R, p->status, st);
    case HAAR_T_BINCSR_F16_U32:
      if (ot != HAAR_OUT_F32 || (lay != HAAR_LAYOUT_SKC && lay != HAAR_LAYOUT_SKC4))
        return set_error(HAAR_ERR_UNSUPPORTED, "%s: BINCSR_F16_U32 needs F32 lighting in SKC or SKC4 layout", who);
      if (lay == HAAR_LAYOUT_SKC4 && !aligned(L, 16))
        return set_error(HAAR_ERR_INVALID_ARG, "%s: SKC4 lighting must be 16-byte aligned", who);
      if (C > 4) return set_error(HAAR_ERR_UNSUPPORTED, "%s: BINCSR supports at most 4 channels", who);
      if (t->bins < 1 || t->bins > 255 || t->K < 1 || t->idx == nullptr || t->bin_of == nullptr)
        return set_error(HAAR_ERR_INVALID_ARG, "%s: BINCSR needs 1..255 bins, K >= 1, idx and bin_of", who);
      return launch_shade_bincsr_f16((const __half*)t->vals, (const uint32_t*)t->idx, t->bin_of, t->V, t->bins,
                                     t->K, S, C, (const float*)L, p->K, lay == HAAR_LAYOUT_SKC4, R, st);
    default:
      return set_error(HAAR_ERR_INVALID_ARG, "%s: unknown transport kind %d", who, t->kind);
  }
}

haar_status_t shade_vertices(haar_shift_plan_t p, const haar_transport_desc_t* t, const void* L, int S,
                             float* R, void* stream) {
  HS_ENTRY("shade_vertices");
  return shade_impl(p, t, L, S, R, (cudaStream_t)stream, "shade_vertices");
}

haar_status_t shade_batch(haar_shift_plan_t p, const float* cin, const double* params, int S,
                          const haar_transport_desc_t* t, float* R, void* stream) {
  HS_ENTRY("shade_batch");
  haar_status_t r = check_shift_args(p, cin, params, S, p ? p->light : nullptr, "shade_batch");
  if (r != HAAR_OK) return r;
  if (t == nullptr || R == nullptr) return set_error(HAAR_ERR_INVALID_ARG, "shade_batch: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  r = launch_setup(p, cin, params, p->light, S, st);
  if (r != HAAR_OK) return r;
  r = (p->desc.kind == HAAR_SHIFT_ROTATE_CHAIN) ? launch_chain(p, params, S, p->light, st)
                                                : launch_shift(p, cin, S, p->light, st);
  if (r != HAAR_OK) return r;
  return shade_impl(p, t, p->light, S, R, st, "shade_batch");
}

haar_status_t haar_transport_group(int V, int N, const int32_t* rowptr, const uint16_t* idx, const float* vals,
                                   int32_t* gptr, uint16_t* gidx, float* gvals, void* stream) {
  HS_ENTRY("haar_transport_group");
  if (V < 0 || N < 1 || N > 65536) return set_error(HAAR_ERR_INVALID_ARG, "haar_transport_group: V=%d N=%d", V, N);
  if (V == 0) return HAAR_OK;
  if (!rowptr || !idx || !gptr || (gidx == nullptr) != (gvals == nullptr) || (gidx && !vals))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_transport_group: null pointer");
  return launch_gcsr_pack(V, N, rowptr, idx, vals, gptr, gidx, gvals, (cudaStream_t)stream);
}

haar_status_t haar_view_bins(int V, int S, int bins, const float* pos, const float* nrm, const float* cams,
                             const float* bin_dirs, uint8_t* bin_of, void* stream) {
  HS_ENTRY("haar_view_bins");
  if (V < 0 || S < 1 || bins < 1 || bins > 255)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_view_bins: bad sizes V=%d S=%d bins=%d", V, S, bins);
  if (V == 0) return HAAR_OK;
  if (!pos || !nrm || !cams || !bin_dirs || !bin_of)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_view_bins: null pointer");
  return launch_view_bins(V, S, bins, pos, nrm, cams, bin_dirs, bin_of, (cudaStream_t)stream);
}

haar_status_t haar_normal_rotations(int V, const float* normals, double* params, void* stream) {
  HS_ENTRY("haar_normal_rotations");
  if (V < 0) return set_error(HAAR_ERR_INVALID_ARG, "haar_normal_rotations: V = %d", V);
  if (V == 0) return HAAR_OK;
  if (!normals || !params) return set_error(HAAR_ERR_INVALID_ARG, "haar_normal_rotations: null pointer");
  if (!aligned(normals, 4) || !aligned(params, 8))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_normal_rotations: misaligned pointer");
  return launch_normal_rotations(V, normals, params, (cudaStream_t)stream);
}

static bool triple_map_ok(int H, int W) { return is_pow2(H) && H >= 2 && (W == H || W == 2 * H); }

long long haar_triple_work_floats(int H, int W, int C) {
  if (!triple_map_ok(H, W) || (long long)H * W > 8192 || C < 1 || C > 4) return -1;
  return triple_work_floats(H, W, C);
}

haar_status_t haar_triple_product(int H, int W, int C, int V, const float* light, const float* brdf,
                                  long long brdf_stride, const float* vis, long long vis_stride, float* out,
                                  float* work, void* stream) {
  HS_ENTRY("haar_triple_product");
  if (!triple_map_ok(H, W))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: map %d x %d (H a power of two >= 2, W = H or 2H)",
                     H, W);
  const long long N = (long long)H * W;
  if (N > 8192)
    return set_error(HAAR_ERR_UNSUPPORTED, "haar_triple_product: N = %lld > 8192 (rows staged in shared memory)", N);
  if (C < 1 || C > 4) return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: C = %d not in [1, 4]", C);
  if (V < 0) return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: V = %d", V);
  if (V == 0) return HAAR_OK;
  if (!light || !brdf || !vis || !out || !work)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: null pointer");
  if (brdf_stride < N || vis_stride < N || brdf_stride % 4 || vis_stride % 4)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: strides %lld, %lld (>= N, multiples of 4)",
                     brdf_stride, vis_stride);
  if (!aligned(brdf, 16) || !aligned(vis, 16) || !aligned(work, 16) || !aligned(light, 4) || !aligned(out, 4))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_triple_product: misaligned pointer");
  return launch_triple(H, W, C, V, light, brdf, brdf_stride, vis, vis_stride, out, work, (cudaStream_t)stream);
}

long long haar_shade_triple_work_floats(int H, int W, int C) {
  if (!triple_map_ok(H, W) || (long long)H * W > 8192 || C < 1 || C > 4) return -1;
  return shade_triple_work_floats(H, W, C);
}

haar_status_t haar_shade_triple(int H, int W, int C, int V, const float* light, const float* brdf_local,
                                const double* params, const float* vis, long long vis_stride, float* out,
                                float* work, void* stream) {
  HS_ENTRY("haar_shade_triple");
  if (!triple_map_ok(H, W))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: map %d x %d (H a power of two >= 2, W = H or 2H)", H, W);
  const long long N = (long long)H * W;
  if (N > 8192)
    return set_error(HAAR_ERR_UNSUPPORTED, "haar_shade_triple: N = %lld > 8192 (rows staged in shared memory)", N);
  if (C < 1 || C > 4) return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: C = %d not in [1, 4]", C);
  if (V < 0) return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: V = %d", V);
  if (V == 0) return HAAR_OK;
  if (!light || !brdf_local || !params || !vis || !out || !work)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: null pointer");
  if (vis_stride < N || vis_stride % 4)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: vis stride %lld (>= N, a multiple of 4)", vis_stride);
  if (!aligned(vis, 16) || !aligned(work, 16) || !aligned(params, 8) || !aligned(light, 4) ||
      !aligned(brdf_local, 4) || !aligned(out, 4))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_triple: misaligned pointer");
  return launch_shade_triple(H, W, C, V, light, brdf_local, params, vis, vis_stride, out, work,
                             (cudaStream_t)stream);
}

haar_status_t haar_rasterize(int V, const float* pos, int T, const int32_t* tris, const float* view_proj, int width,
                             int height, float* screen, unsigned long long* zbuf, int32_t* tri_id, float* bary,
                             void* stream) {
  HS_ENTRY("haar_rasterize");
  if (V < 0 || T < 0 || width < 1 || height < 1 || width > 16384 || height > 16384)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_rasterize: V=%d T=%d image %d x %d", V, T, width, height);
  if ((V > 0 && (!pos || !screen)) || (T > 0 && !tris) || !view_proj || !zbuf || !tri_id || !bary)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_rasterize: null pointer");
  if (!aligned(pos, 4) || !aligned(tris, 4) || !aligned(view_proj, 4) || !aligned(screen, 16) || !aligned(zbuf, 8) ||
      !aligned(tri_id, 4) || !aligned(bary, 8))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_rasterize: misaligned pointer");
  return launch_rasterize(V, pos, T, tris, view_proj, width, height, screen, zbuf, tri_id, bary,
                          (cudaStream_t)stream);
}

haar_status_t haar_shade_pixels(int width, int height, int C, int V, int T, const int32_t* tri_id, const float* bary,
                                const int32_t* tris, const float* vert_rad, const float* background, float* image,
                                void* stream) {
  HS_ENTRY("haar_shade_pixels");
  if (width < 1 || height < 1 || width > 16384 || height > 16384 || C < 1 || C > 64 || V < 0 || T < 0)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_pixels: image %d x %d C=%d V=%d T=%d", width, height, C, V, T);
  if (!tri_id || !bary || (T > 0 && !tris) || (V > 0 && !vert_rad) || !background || !image)
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_pixels: null pointer");
  if (!aligned(bary, 8) || !aligned(tri_id, 4) || !aligned(tris, 4) || !aligned(vert_rad, 4) ||
      !aligned(background, 4) || !aligned(image, 4))
    return set_error(HAAR_ERR_INVALID_ARG, "haar_shade_pixels: misaligned pointer");
  return launch_shade_pixels(width, height, C, V, T, tri_id, bary, tris, vert_rad, background, image,
                             (cudaStream_t)stream);
}

}  // extern "C"
