/*
 * haarshift.h - C ABI of the Haar-domain phase-shift and shading library
 * (sm_103a).
 *
 * What it computes (Alnasser & Foroosh, "Non-Linear Phase-Shifting of Haar
 * Wavelets for Run-Time All-Frequency Lighting"):
 *
 *  - haar_shift: the Haar coefficients of a lat-long lighting map after a
 *    translation (linear phase shift) or a rotation g(theta, phi) =
 *    f(Theta, Phi) (non-linear phase shift, Sec. "Rotating Haar",
 *    Eq. tRot/theta/phi/compfunc), computed from the coefficients of the
 *    original map.
 *  - shade_vertices: the per-vertex light-transport integral as the double
 *    product of shifted lighting coefficients and each vertex's Haar
 *    transport vector (Eq. 1-3 with BRDF x cosine x visibility folded into one
 *    transfer function; Parseval for orthonormal Haar bases).
 *
 * Conventions shared by every entry point
 *  - Map: H x W lat-long map, H = 2^n (1 <= n <= 12), W = H or 2H; rows are
 *    elevation theta_i = (i + 1/2) pi / H, columns azimuth
 *    phi_j = (j + 1/2) 2 pi / W; d = (sin t sin p, cos t, sin t cos p), Y up.
 *  - Haar: orthonormal non-standard 2-D Haar.  On 2x2 blocks (a b / c d):
 *    A = (a+b+c+d)/2, H = (b+d-a-c)/2, V = (c+d-a-b)/2, D = (a+d-b-c)/2.
 *    Canonical order of the N = H W coefficients: A_n (W/H values), then for
 *    l = n..1 the bands H_l, V_l, D_l, each row-major; band b of level l
 *    occupies [g (1+b), g (2+b)) with g = (W/H) 4^(n-l).
 *  - Resampling: bilinear between pixel centres of the map extended across
 *    its borders: azimuth cyclic; SPHERE: a row beyond a pole is the mirrored
 *    row half a turn away; TORUS: rows cyclic.
 *  - Memory: every pointer argument is caller-owned device memory unless a
 *    comment says otherwise; the library never frees caller memory.  Plans
 *    own their workspace (allocated in haar_shift_plan, freed in
 *    haar_shift_plan_destroy).
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Compute entry points are asynchronous, allocate nothing and do not
 *    synchronise; a plan's workspace is shared by all calls on that plan,
 *    so calls on one plan must be ordered (same stream, or synchronised).
 *  - Errors: arguments are validated before any launch; a failing call
 *    returns a non-zero haar_status_t and haar_last_error() (thread-local)
 *    describes it.  Setting the environment variable HAAR_FAULT_INJECT to an
 *    entry point's name makes that entry point return HAAR_ERR_INJECTED
 *    before launching anything (host-side fault injection for tests).
 */
#ifndef HAARSHIFT_H
#define HAARSHIFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HAAR_API __attribute__((visibility("default")))
#else
#define HAAR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HAAR_OK = 0,
  HAAR_ERR_INVALID_ARG = 1, /* bad size, null pointer, misalignment, bad enum */
  HAAR_ERR_UNSUPPORTED = 2, /* valid but not implemented combination */
  HAAR_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  HAAR_ERR_TIMEOUT = 4,     /* a device-side bounded wait gave up */
  HAAR_ERR_INJECTED = 5,    /* HAAR_FAULT_INJECT named this entry point */
  HAAR_ERR_NOMEM = 6        /* workspace allocation failed */
} haar_status_t;

typedef enum {
  HAAR_SHIFT_TRANSLATE = 0,   /* params [S][2] float64: (dx, dy) in pixels */
  HAAR_SHIFT_ROTATE = 1,      /* params [S][9] float64: R row-major, p' = R p; R must be a
                                 rotation (orthonormal, det +1) or a positive multiple of one:
                                 the kernels use its factorisation Ry(a) Rx(b) Ry(c) */
  HAAR_SHIFT_ROTATE_EULER = 2, /* params [S][3] float64: (alpha, beta, gamma),
                                 R = Rz(gamma) Ry(beta) Rx(alpha) (Eq. tRot) */
  HAAR_SHIFT_ROTATE_CHAIN = 3  /* params as ROTATE_EULER; the paper's own route, an
                                 approximation: the rotated map's finest derivative
                                 fields by the chain rule (Eq. pde1-pde3, the mixed
                                 term's second-order rule completed) and the detail
                                 coefficients from them by Eq. conv / tker / sker;
                                 float32 output only; the plan holds C x 4 x N floats
                                 of fields per shift */
} haar_shift_kind_t;

typedef enum { HAAR_BOUNDARY_SPHERE = 0, HAAR_BOUNDARY_TORUS = 1 } haar_boundary_t;

typedef enum {
  HAAR_OUT_F32 = 0,       /* float32 */
  HAAR_OUT_BF16_HILO = 1, /* two bfloat16 planes: hi = bf16(x), lo = bf16(x - hi);
                             the lo plane follows the hi plane (S*C*K elements) */
  HAAR_OUT_F16 = 2        /* IEEE binary16 */
} haar_out_t;

typedef enum {
  HAAR_LAYOUT_SCK = 0, /* out[s][c][k] */
  HAAR_LAYOUT_SKC = 1, /* out[s][k][c]  (channels interleaved) */
  HAAR_LAYOUT_KSC = 2, /* out[k][s][c]  (coefficient-major) */
  HAAR_LAYOUT_SKC4 = 3 /* out[s][k][4]: SKC with the channel axis padded to 4 (C <= 4; the
                          pad entries are not written), so a coefficient's channels are one
                          16-byte vector for gathers */
} haar_layout_t;

typedef struct haar_shift_plan_s* haar_shift_plan_t;

typedef struct {
  int height;     /* H = 2^n */
  int width;      /* W in {H, 2H} */
  int channels;   /* C, 1..64 */
  int kind;       /* haar_shift_kind_t */
  int boundary;   /* haar_boundary_t */
  int max_shifts; /* largest S any call on this plan will pass (workspace size) */
  int out_coeffs; /* K: the K lowest canonical coefficients are written (0 = all) */
  int out_type;   /* haar_out_t */
  int out_layout; /* haar_layout_t */
  int start_level; /* k >= 0, H >> k >= 2: the shift starts at level k (Sec. "Algorithmic
                      optimization"): it is taken of the level-k scaling image, the
                      (H/2^k) x (W/2^k) map of 2^k x the 2^k x 2^k block means, whose
                      coefficients are the N/4^k coarsest of coeffs_in; a translation
                      moves it by (dx, dy)/2^k, a rotation is unchanged.  Only those
                      N/4^k coefficients are produced (K <= N/4^k; out_coeffs = 0 means
                      all of them), for O(N/4^k) work.  0 = the full map. */
} haar_shift_desc_t;

/* Create a plan: validates the descriptor and allocates its device workspace
 * (pixel map C*H*W floats, per-shift tables and counters, shade_batch's
 * lighting buffer) on the current device.  Translation plans with float32
 * SCK output of all N coefficients, H >= 64 and max_shifts * (H/64)(W/64) >=
 * 2432 also hold the map extended by one period of rows plus 65 and by 68
 * columns (C*(2H+65)*(W+68) floats for SPHERE, C*(H+65)*(W+68) for TORUS),
 * from which their batch kernel stages each tile's window by TMA.  *out
 * receives the plan. */
HAAR_API haar_status_t haar_shift_plan(const haar_shift_desc_t* desc, haar_shift_plan_t* out);

/* Release a plan and its workspace (synchronises the device first). */
HAAR_API haar_status_t haar_shift_plan_destroy(haar_shift_plan_t plan);

/* Device-side status of the plan's kernels since the last reset: bit
 * (1 << HAAR_ERR_TIMEOUT) is set when a bounded wait of a pipelined kernel
 * (tensor-core contraction, group-CSR shading) gave up; that launch's
 * radiance is then incomplete.  Synchronises the device; *status_out
 * receives the bits (0 = fine); reset != 0 clears them. */
HAAR_API haar_status_t haar_shift_plan_status(haar_shift_plan_t plan, int* status_out, int reset);

/* The phase shift (Sec. "Rotating Haar" and "Mathematical description";
 * Sec. "Algorithmic optimization" for the O(N) cost):
 *   coeffs_out[s] = Haar( resample_s( Haar^-1(coeffs_in) ) ),  s = 0..S-1.
 * coeffs_in : [C][N] float32, canonical order.
 * params    : device float64, layout given by the plan's kind (see
 *             haar_shift_kind_t); translations may be any real numbers.
 * S         : 1..max_shifts.
 * coeffs_out: K coefficients per (s, c) in the plan's out_type and layout.
 * Integer shifts whose components are multiples of a level's block side 2^l
 * reproduce that level's coefficients as an exact signed permutation of the
 * input (bit-for-bit).  Uses the plan workspace: calls on one plan must not
 * overlap on the GPU. */
HAAR_API haar_status_t haar_shift(haar_shift_plan_t plan, const float* coeffs_in, const double* params,
                         int S, void* coeffs_out, void* stream);

/* The phase shift of haar_shift without a plan and without allocating.
 * (The paper has no counterpart; this is a calling convenience.)  For callers
 * that cannot allocate device memory at all: plug-ins inside a host renderer
 * or engine whose device memory belongs to the host's own allocator, and
 * real-time frame loops that may not call cudaMalloc/cudaFree, which
 * synchronise the device.  It computes exactly what haar_shift computes for
 * the same descriptor (desc->max_shifts is ignored; S is this call's count)
 * and calls no cudaMalloc, cudaFree or allocating library routine: its
 * scratch is one fixed array of 2 Mi floats (8 MiB) in the library's device
 * memory, which every GPU that loads the library holds until the process
 * exits.  A call needs, each part rounded up to a multiple of 64 floats:
 * the pixel map (C*H*W floats for translations, 8*H*W*ceil(C/3) for
 * rotations), 4*(H+W) floats of tables, for rotations S*8*(H+W) floats of
 * per-rotation tables, 20*S floats of shift records, S*C*T floats of tile
 * means (T = H*W/4096 tiles for H >= 64, 1 or 2 below; T = H*W/256 for
 * float32 KSC translations) and S tile counters, for the map the shift runs
 * on (H, W after start_level).  So RGB 256x512 takes up to 166 rotations or
 * ~14 500 SCK translations, RGB 128x256 up to ~4 900 KSC translations, and
 * RGB 1024x2048 does not fit.  Larger calls are rejected with
 * HAAR_ERR_INVALID_ARG and a message giving both sizes.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the life
 * of the process (a device reset after that first call is not supported);
 * make that first call before any stream capture.  Every call on a device shares the one array
 * and it keeps the previous call's contents (the call clears the tile
 * counters it needs at zero itself): calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results; order them.
 * coeffs_in, params, coeffs_out: as for haar_shift (device memory). */
HAAR_API haar_status_t haar_shift_noalloc(const haar_shift_desc_t* desc, const float* coeffs_in,
                                          const double* params, int S, void* coeffs_out, void* stream);

/* Forward orthonormal Haar transform of `batch` H x W float32 maps
 * ([batch][H][W] row-major) into [batch][N] canonical coefficients; `scale`
 * multiplies every output (1.0 for the plain transform). */
HAAR_API haar_status_t haar_forward(int H, int W, int batch, const float* maps, float* coeffs, float scale,
                           void* stream);

/* Inverse transform: [batch][N] coefficients -> [batch][H][W] maps. */
HAAR_API haar_status_t haar_inverse(int H, int W, int batch, const float* coeffs, float* maps,
                           void* stream);

typedef enum {
  HAAR_T_DENSE_F32 = 0,     /* vals [V][K] float32, lowest K coefficients */
  HAAR_T_DENSE_BF16 = 1,    /* vals [V][K] bfloat16, lowest K coefficients */
  HAAR_T_CSR_F32_U16 = 2,   /* vals float32, idx uint16, rowptr int32 [V+1] */
  HAAR_T_BINCSR_F16_U32 = 3, /* vals [V][bins][K] binary16, idx [V][bins][K] uint32,
                               bin_of [S][V] uint8 selects the bin of (s, v) */
  HAAR_T_GCSR_F32_U16 = 4    /* vertex-group CSR made by haar_transport_group: groups of
                               HAAR_GCSR_GROUP consecutive vertices share one sorted
                               union index list idx (uint16) with values
                               [nnz][HAAR_GCSR_GROUP] float32 (0 where a vertex lacks
                               the coefficient); rowptr = group offsets
                               [ceil(V/HAAR_GCSR_GROUP) + 1] int32 */
} haar_transport_kind_t;

/* vertices per group of HAAR_T_GCSR_F32_U16 */
#define HAAR_GCSR_GROUP 4

typedef struct {
  int kind;                    /* haar_transport_kind_t */
  int V;                       /* vertices */
  int K;                       /* dense: coefficients per row; BINCSR: entries per bin */
  int bins;                    /* BINCSR only */
  const void* vals;            /* device */
  const void* idx;             /* device (CSR, BINCSR) */
  const int32_t* rowptr;       /* device (CSR) */
  const uint8_t* bin_of;       /* device (BINCSR) */
} haar_transport_desc_t;

/* The double product (Eq. 2-5 with two factors, Parseval):
 *   radiance[v][s][c] = sum_k T[v][k] * L'[s][c][k].
 * lighting: the output of haar_shift on this plan (its out_type/layout).
 * Supported pairings (others return HAAR_ERR_UNSUPPORTED):
 *   DENSE_F32        with F32  lighting, layout SCK, K <= plan K;
 *   DENSE_BF16       with BF16_HILO lighting, layout SCK, K == plan K,
 *                    K % 64 == 0 (tcgen05 tensor-core GEMM, FP32 accumulate,
 *                    T x L_hi + T x L_lo);
 *   CSR_F32_U16      with F32  lighting, layout KSC (S*C % 4 == 0);
 *   BINCSR_F16_U32   with F32  lighting, layout SKC or SKC4;
 *   GCSR_F32_U16     with F32  lighting, layout KSC (S*C % 4 == 0).
 * radiance: [V][S][C] float32, overwritten.  It may also be page-locked host
 * memory mapped into the device's address space (cudaHostAlloc'd, unified
 * addressing): the shading kernels write it with plain stores, so the result
 * reaches the host over the host link (NVLink-C2C on Grace-Blackwell) without
 * a separate device-to-host copy.  Launches that use the same plan must be
 * ordered (one stream, or events): the plan's workspace and device counters
 * are shared. */
HAAR_API haar_status_t shade_vertices(haar_shift_plan_t plan, const haar_transport_desc_t* transport,
                             const void* lighting, int S, float* radiance, void* stream);

/* haar_shift followed by shade_vertices, with the shifted lighting kept in
 * the plan's workspace (stream-ordered, no host synchronisation). */
HAAR_API haar_status_t shade_batch(haar_shift_plan_t plan, const float* coeffs_in, const double* params,
                          int S, const haar_transport_desc_t* transport, float* radiance,
                          void* stream);

/* Repack top-K CSR transport (rows sorted by index, rowptr int32 [V+1],
 * idx uint16, vals float32) into the vertex-group CSR of HAAR_T_GCSR_F32_U16:
 * the union of the indices of every HAAR_GCSR_GROUP (G) consecutive rows,
 * sorted, with the values of each row at its union positions (0 elsewhere).
 * A storage form of the top-K (non-linear) approximation cited in Sec.
 * "Haar-domain methods": the double product is unchanged, each lighting row
 * gathered serves G vertices.  N: coefficients per map (<= 65536; indices
 * >= N are dropped).  gptr [ceil(V/G) + 1] int32 (device) receives the group
 * offsets; gptr[ceil(V/G)] is the total.  Call once with gidx = gvals = NULL
 * to get gptr, then again with gidx [total] uint16 and gvals [total][G]
 * float32 (16-byte aligned). */
HAAR_API haar_status_t haar_transport_group(int V, int N, const int32_t* rowptr, const uint16_t* idx,
                                            const float* vals, int32_t* gptr, uint16_t* gidx, float* gvals,
                                            void* stream);

/* View-bin selection for view-dependent transport (the paper's per-pixel
 * "BRDF tile id" of the rotation input pass, Sec. "Experimental results"):
 * for every (s, v) the bin whose local direction has the largest dot product
 * with the vertex's local view direction normalize(cam[s] - pos[v]),
 * expressed in the frame (b1, b2, n) of the branchless orthonormal basis of
 * Duff et al. 2017; ties keep the lower bin.  pos, nrm: [V][3] float32;
 * cams: [S][3] float32; bin_dirs: [bins][3] float32 (local, z = normal);
 * bin_of: [S][V] uint8 (bins <= 255). */
HAAR_API haar_status_t haar_view_bins(int V, int S, int bins, const float* pos, const float* nrm,
                             const float* cams, const float* bin_dirs, uint8_t* bin_of,
                             void* stream);

/* ---------------------------------------------------------------------------
 * The paper's shading loop (Sec. "Algorithmic optimization" and Sec.
 * "Experimental results": rotation input pass, rotation pass, triple
 * integral pass): each vertex's BRDF map, given in a local frame whose normal
 * sits at the +y pole, is rotated onto the vertex normal with haar_shift
 * (HAAR_SHIFT_ROTATE, parameters from haar_normal_rotations), then the
 * outgoing radiance is the triple product of lighting x rotated BRDF x
 * visibility (Sec. "Related work", Tripling Coefficient Theorem).
 * ------------------------------------------------------------------------- */

/* Rotation records of the rotation input pass: for normals [V][3] float32
 * (normalised here) params [V][9] float64 receives R = Rx(-theta_N)
 * Ry(-phi_N), row-major, theta_N = acos(n_y), phi_N = atan2(n_x, n_z): a tilt
 * about the x axis and a shift along phi, with R N = +y.  As
 * HAAR_SHIFT_ROTATE parameters (g(w) = f(R w)) it carries a local-frame map
 * onto the normal.  A zero normal gives a NaN record. */
HAAR_API haar_status_t haar_normal_rotations(int V, const float* normals, double* params, void* stream);

/* Floats of the workspace haar_triple_product needs for C lighting channels
 * of an H x W map (the lighting's mean over every Haar square, its details
 * and mean packed per square, and a status word). */
HAAR_API long long haar_triple_work_floats(int H, int W, int C);

/* The Haar triple product of the triple integral pass:
 *   out[v][c] = sum_ijk C_ijk light[c][i] brdf[v][j] vis[v][k]
 * with the tripling coefficients of the orthonormal basis above (unit pixel
 * measure: 1/H for three scaling functions, 1/B for the three distinct
 * wavelet types on one square of side B, and for a repeated wavelet the value
 * of the third basis function on its square), evaluated square by square in
 * O(N) per vertex with the factors' means over each square.  This equals the
 * pixel sum of the three reconstructed maps; fold the solid-angle weight
 * sin(theta) dtheta dphi into one factor (visibility) for the integral over
 * the sphere.
 *   light: [C][N] float32, 1 <= C <= 4;  brdf, vis: row v at brdf + v *
 *   brdf_stride (floats), canonical order, 16-byte aligned rows (strides a
 *   multiple of 4); out: [V][C] float32; work: haar_triple_work_floats(H, W,
 *   C) floats, 16-byte aligned.  Needs N = H W <= 8192 (both factors of a
 *   vertex are staged in shared memory by bulk copies).  After the call, the
 *   int at work[0] is 0, or has bit HAAR_ERR_TIMEOUT set if a bulk copy did
 *   not complete within 2 s (that vertex's outputs are then NaN). */
HAAR_API haar_status_t haar_triple_product(int H, int W, int C, int V, const float* light, const float* brdf,
                                           long long brdf_stride, const float* vis, long long vis_stride,
                                           float* out, float* work, void* stream);

/* Floats of the workspace haar_shade_triple needs (lighting means, the
 * BRDF's pixel map, angle tables and a status word). */
HAAR_API long long haar_shade_triple_work_floats(int H, int W, int C);

/* The rotation pass and the triple integral pass fused, one CTA per vertex:
 *   out[v][c] = sum_ijk C_ijk light[c][i] b_v[j] vis[v][k],
 * b_v = the coefficients of the local-frame BRDF map brdf_local [N] after the
 * rotation record params[v] (HAAR_SHIFT_ROTATE semantics, SPHERE boundary:
 * g(w) = f(R w), bilinear).  The same result as haar_shift (one channel, one
 * shift per vertex) followed by haar_triple_product, without writing the
 * rotated BRDF to memory.  light: [C][N]; params: [V][9] float64 (e.g. from
 * haar_normal_rotations); vis rows as in haar_triple_product; out: [V][C];
 * work: haar_shade_triple_work_floats(H, W, C) floats, 16-byte aligned, the
 * int at work[0] the status word as in haar_triple_product.  N <= 8192. */
HAAR_API haar_status_t haar_shade_triple(int H, int W, int C, int V, const float* light, const float* brdf_local,
                                         const double* params, const float* vis, long long vis_stride, float* out,
                                         float* work, void* stream);

/* ---------------------------------------------------------------------------
 * Headless rasterisation (the paper's rasterisation pass, Sec. "Experimental
 * results", without a graphics API): a fragment buffer of the nearest
 * triangle and its perspective-correct barycentrics per pixel, then per-pixel
 * shading from per-vertex radiance.
 * ------------------------------------------------------------------------- */

/* pos: [V][3] float32; tris: [T][3] int32 vertex indices (a triangle with an
 * index outside [0, V) is dropped); view_proj: 16 float32, row-major,
 * device.  Each vertex is projected as clip = M [x y z 1], ndc = clip / w,
 * screen = ((ndc_x + 1) / 2 width, (1 - ndc_y) / 2 height), rows growing
 * downwards.  A triangle with a vertex at w <= 1e-6 is dropped (no near-plane
 * clipping).  Pixel (px, py) samples its centre (px + 1/2, py + 1/2).  It is
 * covered when the edge functions, oriented to a positive screen area, are
 * > 0, or = 0 on an edge whose direction has dy > 0, or dy = 0 and dx < 0.
 * That rule covers an edge shared by two triangles once.  Depth = (ndc z
 * interpolated + 1) / 2 must lie in [0, 1]; the nearest fragment wins, and on
 * equal depth the lower triangle id.  These decisions are float32 with a
 * fixed operation order and no fused multiply-add.
 * Outputs, for an image of width x height pixels (row-major):
 *   tri_id [H][W] int32, -1 where nothing is hit;
 *   bary [H][W][2] float32, the weights of the triangle's vertices 1 and 2
 *     (vertex 0 gets 1 - b1 - b2), perspective-correct;
 *   screen [V][4] float32 (16-byte aligned) and zbuf [H][W] uint64 are
 *     scratch (zbuf: depth bits << 32 | triangle id). */
HAAR_API haar_status_t haar_rasterize(int V, const float* pos, int T, const int32_t* tris, const float* view_proj,
                                      int width, int height, float* screen, unsigned long long* zbuf,
                                      int32_t* tri_id, float* bary, void* stream);

/* image [H][W][C] float32 = the barycentric interpolation of vert_rad [V][C]
 * over each pixel's triangle (from haar_rasterize), background [C] where
 * tri_id is -1 or not a valid triangle of tris [T][3]. */
HAAR_API haar_status_t haar_shade_pixels(int width, int height, int C, int V, int T, const int32_t* tri_id,
                                         const float* bary, const int32_t* tris, const float* vert_rad,
                                         const float* background, float* image, void* stream);

/* ---------------------------------------------------------------------------
 * Transport surrogate (not in the paper; a learned stand-in for stored
 * transport).  A 4 x 256 GELU MLP (tanh-form GELU) maps a vertex's position, normal and view
 * direction to its transport coefficients at a fixed set of 512 canonical
 * indices (standardised: T_j = mu_j + sigma_j out_j).  Encoding of the 9
 * inputs (position p, normal n, view w) with w_f = pi 2^(f/2), f = 0..15:
 * columns 0..199 = [p, n], per f sin(w_f [p, n]), cos(w_f [p, n]), 2 zeros;
 * columns 200..298 = w, per f sin(w_f w), cos(w_f w); zeros to 320.
 * Flat FP32 parameter vector (haar_mlp_param_count() floats):
 * W1[256][320] b1[256] W2[256][256] b2 W3 b3 W4 b4 Wo[512][256] bo[512].
 * Forward and backward run as bf16 tcgen05 GEMMs with FP32 accumulation;
 * master weights and Adam state are FP32.  A surrogate owns its device
 * buffers (allocated by haar_mlp_create); compute calls allocate nothing and
 * calls on one surrogate must be ordered.
 * ------------------------------------------------------------------------- */
typedef struct haar_mlp_s* haar_mlp_t;

/* Number of floats in the flat parameter vector. */
HAAR_API long long haar_mlp_param_count(void);

/* Create a surrogate: training batches up to max_batch rows and inference in
 * chunks of max_rows rows (both multiples of 128), up to max_groups shifts.
 * Parameters start at zero: set them with haar_mlp_set_params. */
HAAR_API haar_status_t haar_mlp_create(int max_batch, int max_rows, int max_groups, haar_mlp_t* out);
HAAR_API haar_status_t haar_mlp_destroy(haar_mlp_t mlp);

/* Copy the flat FP32 parameters in (any device- or host-accessible pointer,
 * cudaMemcpyDefault) and reset the Adam state; or copy them out. */
HAAR_API haar_status_t haar_mlp_set_params(haar_mlp_t mlp, const float* params, void* stream);
HAAR_API haar_status_t haar_mlp_get_params(haar_mlp_t mlp, float* params, void* stream);

/* out [B][512] float32 = network output for raw inputs [B][9]
 * (position, normal, view direction); B a multiple of 128, <= max_batch. */
HAAR_API haar_status_t haar_mlp_forward(haar_mlp_t mlp, const float* raw, int B, float* out, void* stream);

/* Gradients of the mean squared error against target [B][512] into grads
 * (flat, haar_mlp_param_count() floats; may be NULL) and the loss into
 * loss[0] (device; may be NULL). */
HAAR_API haar_status_t haar_mlp_grads(haar_mlp_t mlp, const float* raw, const float* target, int B, float* grads,
                                      float* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * mean squared error of batch (raw, target); loss[0] (device, may be NULL)
 * receives the batch loss before the step. */
HAAR_API haar_status_t haar_mlp_train_step(haar_mlp_t mlp, const float* raw, const float* target, int B, float lr,
                                           float* loss, void* stream);

/* Surrogate shading, fused: for every (s, v) the network evaluates the
 * transport at the index set from (pos[v], nrm[v], normalize(cams[s] - pos[v]))
 * and the last hidden layer's epilogue takes the double product with the
 * shifted lighting, the output layer folded into the lighting per shift:
 *   radiance[v][s][c] = sum_j (mu_j + sigma_j out_j) L(s, c, idx_j),
 * L(s, c, k) = lighting[s * st_s + c * st_c + k * st_k] (float32, e.g. the
 * output of haar_shift).  pos, nrm [V][3]; cams [S][3]; mu, sigma [512];
 * idx [512] int32; C <= 4; radiance [V][S][C] float32. */
HAAR_API haar_status_t haar_mlp_shade(haar_mlp_t mlp, int V, int S, const float* pos, const float* nrm,
                                      const float* cams, const float* mu, const float* sigma, const int32_t* idx,
                                      const float* lighting, int C, long long st_s, long long st_c, long long st_k,
                                      float* radiance, void* stream);

/* Copy and clear the surrogate's device status word (bit HAAR_ERR_TIMEOUT set
 * when a bounded wait inside a tensor-core kernel gave up). Synchronous. */
HAAR_API haar_status_t haar_mlp_status(haar_mlp_t mlp, int* out);

/* Message describing the last failure on the calling thread ("" if none). */
HAAR_API const char* haar_last_error(void);

/* Library version string. */
HAAR_API const char* haar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HAARSHIFT_H */
