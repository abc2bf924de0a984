/*
 * scw.h -- C ABI of libscw, GB300 (sm_103a) volumetric field synthesis for the
 * coupled-wave method of Sun, Reddy and Mayerich, "sCWatter: open source
 * coupled wave scattering simulation for spectroscopy and microscopy"
 * (arXiv 2404.07293).
 *
 * What the library computes (paper Sec. 2.3, 2.6 and 4.1):
 *   For every output plane z and every Fourier order m = (u, v), the per-plane
 *   spectrum S_c[m](z) of the electric field (c = x, y, z), and then the field
 *       E_c(x_i, y_j, z) = sum_m S_c[m](z) exp(2 pi i (u_m x_i / X + v_m y_j / Y))   (Eq. 10)
 *   on the pixels x_i = x0 + i X/Fx, y_j = y0 + j Y/Fy (one lateral period).
 *   Inside layer l (z_{l-1} <= z < z_l; the last layer also takes z = z_L):
 *       S(z) = W_l (alpha_l o g(z)),  g_j = exp(i k gamma_j (z - z_ref,j)),      (Eq. 30-31, 34)
 *   where k = 2 pi / lambda, modes j in [0, 2M) are forward (z_ref = z_{l-1})
 *   and modes j in [2M, 4M) are backward (z_ref = z_l); W_l holds the E-field
 *   rows of the layer's eigenvectors (rows c*M + m; the E_z rows already carry
 *   the Psi convolution of Eq. 33).
 *   Above the sample (z < z0) and below it (z > z_L), with flag SCW_FLAG_EXTERIOR:
 *       S = p_inc exp(i k s_t (z - z_inc)) + p_ref exp(-i k s_t (z - z0))          (Eq. 9)
 *       S = p_trn exp(i k s_b (z - z_L))
 *   with s_t = s_z(n_top), s_b = s_z(n_bot) from Eq. 2 on the decaying branch.
 *
 * Orders (Sec. 2.2): u in [-floor(U/2), floor((U-1)/2)], likewise v, flat
 * index m = (v + floor(V/2)) U + (u + floor(U/2)); s_x = lambda u / X,
 * s_y = lambda v / Y (Eq. 6).
 *
 * Conventions for every entry point:
 *   - complex64 is two packed floats (re, im); complex128 two packed doubles.
 *   - "DEVICE" pointers are CUDA global memory on the current device; "HOST"
 *     pointers are ordinary (ideally pinned) host memory.
 *   - The caller owns every buffer it passes and keeps it alive until the work
 *     queued on the stream has finished. A plan owns its own workspace and
 *     frees it in scw_plan_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All GPU work is asynchronous on that stream; no entry point except
 *     scw_plan_check, scw_synthesize_host and plan creation synchronises.
 *   - Errors are returned as scw_status, with a message in scw_last_error()
 *     (thread-local). Nothing traps on the device: kernels record problems in
 *     a device error word that scw_plan_check reads back.
 *   - There is no CPU fallback: without a usable sm_103a device every entry
 *     point that would launch work returns SCW_ERR_CUDA.
 */
#ifndef SCW_H
#define SCW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scw_plan_s* scw_plan_t;

typedef enum {
  SCW_OK = 0,
  SCW_ERR_INVALID_ARGUMENT = 1, /* a size, pointer or value is out of range       */
  SCW_ERR_UNSUPPORTED = 2,      /* valid but not handled by this build           */
  SCW_ERR_OUT_OF_MEMORY = 3,    /* a workspace allocation failed                 */
  SCW_ERR_CUDA = 4,             /* a CUDA runtime/driver call failed             */
  SCW_ERR_TIMEOUT = 5,          /* a device-side bounded wait ran out            */
  SCW_ERR_NUMERIC = 6,          /* non-finite value detected                     */
  SCW_ERR_STATE = 7,            /* call order violated (e.g. no layers set)     */
  SCW_ERR_BOUNDS = 8            /* SCW_FLAG_DEBUG_BOUNDS: an index left its buffer */
} scw_status;

/* Arithmetic of the mode contraction (the other steps are FP64-argument /
 * FP32-value phases and an FP32 inverse FFT in every mode). */
typedef enum {
  SCW_PREC_FP32 = 0,        /* FP32 SIMT complex GEMM (the plain path)                 */
  SCW_PREC_SPLIT_BF16 = 1,  /* tcgen05: W = hi + lo (BF16), C = hi + lo, 3 products,
                               FP32 accumulation in tensor memory                       */
  SCW_PREC_FP16 = 2         /* tcgen05: W in FP16, C = hi + lo (FP16), 2 products      */
} scw_precision;

enum {
  SCW_FLAG_EXTERIOR = 1u, /* planes outside [z0, z_L] allowed (needs p_inc/p_ref/p_trn) */
  SCW_FLAG_HOST_IO = 2u,  /* plan also owns device copies of W/gamma/alpha/p for
                             scw_synthesize_host                                        */
  SCW_FLAG_AUTOTUNE = 4u, /* time the best contraction schedules on the device at plan
                             creation (otherwise a makespan model picks the split);
                             results are cached per device and problem shape           */
  SCW_FLAG_DEBUG_BOUNDS = 8u /* index checks: every kernel of the plan compares each global
                             index it forms (spectra, x-pass rows, twiddles, B operand,
                             gamma/alpha, the FP32 path's operands, the field) with the
                             extent of its buffer; an index outside is not accessed, the
                             device error word records it and scw_plan_check returns
                             SCW_ERR_BOUNDS. The bulk copies of the tensor-core contraction
                             are driven by a task table built on the host: plan creation
                             checks every task's W, B and partial-spectrum ranges against
                             their allocations and fails with SCW_ERR_BOUNDS. Results are
                             the same as without the flag; the checks cost a compare per
                             access or per loop                                         */
};

typedef struct {
  int U, V, L;              /* orders along x and y (M = U V), number of layers        */
  double lambda, X, Y;      /* vacuum wavelength and lateral period, same length unit   */
  const double* z_bounds;   /* HOST [L+1], strictly ascending z_0 .. z_L                */
  int Fx, Fy, Fz;           /* output grid: Fx, Fy multiples of 8 in [8, 4096]; Fz >= 1 */
  const double* z_planes;   /* HOST [Fz], non-decreasing                                 */
  double x0, y0;            /* position of output pixel (0, 0)                          */
  double n_top;             /* real refractive index above the sample                   */
  double n_bot_re, n_bot_im;/* complex refractive index below the sample                */
  double z_inc;             /* plane at which p_inc is given (the paper's z-bar)        */
  int precision;            /* scw_precision                                             */
  unsigned flags;           /* SCW_FLAG_*                                                */
  int k_split;              /* contraction split along the 4M modes; 0 = choose         */
  int illuminations;        /* I incident fields sharing this solve (0 counts as 1): the
                               modes (W, gamma) are read once per layer for all of them, alpha
                               is [I][L][4M], p_inc/p_ref/p_trn are [I][3][M] and the field is
                               [I][3][Fz][Fy][Fx]; I Fz <= 65535                            */
  double pupil_na;          /* > 0: below the sample only the orders with |s_bar| <= pupil_na
                               pass (the numerical aperture of a collecting objective, in the
                               units of s_bar = lambda (u/X, v/Y)); 0: no pupil             */
  int tiles_x, tiles_y;     /* periodic tiling (0 counts as 1, at most 64 each): the field covers
                               tiles_x x tiles_y lateral periods, (tiles_y Fy) x (tiles_x Fx)
                               pixels; the unit cell is computed once and stored to every
                               tile, since E(x + a X, y + b Y) = E(x, y) (Eq. 10)          */
  long long out_ld;         /* row pitch of the field in complex elements, even; 0 means
                               tiles_x Fx. With out_plane_stride it lets the field of a plan (or
                               of each batched item) be written as a patch of a larger
                               mosaic: pixel (x, y) of plane slice s goes to
                               out[s out_plane_stride + y out_ld + x]                     */
  long long out_plane_stride; /* complex elements between consecutive plane slices
                               s = (i 3 + c) Fz + f, even; 0 means tiles_y Fy out_ld. The
                               field pointer must be 16-byte aligned (16-byte stores)       */
} scw_desc;

typedef struct {
  int M;                    /* U V                                                       */
  int active_layers;        /* layers that hold at least one plane                       */
  int planes_per_layer_pad; /* plane slots per layer in the contraction (multiple of 8)  */
  int k_split;              /* split actually used                                       */
  int exterior_planes;      /* planes outside [z0, z_L]                                  */
  size_t workspace_bytes;   /* device bytes owned by the plan                            */
  double convert_ms;        /* GPU time of the last W conversion (scw_plan_set_layers)   */
  int kernels_per_synthesis;/* kernel launches queued by one scw_synthesize              */
  int items;                /* 1, or the batch size                                      */
  int contract_ctas;        /* persistent CTAs of the tensor-core contraction            */
  int contract_tasks;       /* (item, unit, row tile, split) tasks they share            */
  double schedule_max_load; /* longest CTA's work in K-stages (+2 per task)              */
  double schedule_mean_load;/* mean CTA work in the same unit                            */
} scw_plan_info;

/* Validate `desc`, assign planes to layers (Sec. 2.6.2: half-open layers, the
 * last one closed), build the order/twiddle tables of the orders (Sec. 2.2)
 * and the output grid (Eq. 10) and allocate the workspace. The table uploads,
 * workspace clears and (with SCW_FLAG_AUTOTUNE) the timed contraction
 * candidates are queued on `stream` (a cudaStream_t; NULL = the legacy default
 * stream), so they are ordered after the caller's earlier work there; the
 * call synchronises `stream` before it returns. On success *out owns the
 * workspace.
 * Errors: INVALID_ARGUMENT (sizes, non-ascending z, planes outside [z0,z_L]
 * without SCW_FLAG_EXTERIOR), UNSUPPORTED (sizes above the build's limits),
 * OUT_OF_MEMORY, CUDA (no sm_103a device). */
scw_status scw_plan(const scw_desc* desc, void* stream, scw_plan_t* out);
/* scw_plan on the legacy default stream. */
scw_status scw_plan_create(const scw_desc* desc, scw_plan_t* out);

/* Free everything the plan owns. NULL is accepted. */
scw_status scw_plan_destroy(scw_plan_t plan);

/* Attach the solved layers (the output of the connection-equation solve,
 * Sec. 2.5.4 and Sec. 4.1's per-layer precompute):
 *   W      DEVICE complex64  [L][3M][4M] row-major, rows c*M + m
 *   gamma  DEVICE complex128 [L][4M]  modes [0,2M) forward, [2M,4M) backward
 *   alpha  DEVICE complex128 [L][4M]
 *   p_inc, p_ref, p_trn  DEVICE complex128 [3][M], required with
 *          SCW_FLAG_EXTERIOR, otherwise may be NULL
 * The plan keeps gamma/alpha/p pointers (not copies) and converts W once into
 * the layout of the chosen precision (split-BF16 hi/lo, FP16, or the
 * transposed FP32 copy), queued on `stream`. W itself is not kept. */
scw_status scw_plan_set_layers(scw_plan_t plan, const void* W, const void* gamma,
                               const void* alpha, const void* p_inc, const void* p_ref,
                               const void* p_trn, void* stream);

/* The whole hot path: phases (a), contraction (b), inverse FFT (c).
 *   out  DEVICE complex64 [3][Fz][Fy][Fx], x fastest (component-major).
 * The first call for a given `out` launches the kernels and captures them into
 * a CUDA graph; later calls with the same `out` replay the graph (one launch).
 * scw_plan_set_layers and scw_plan_set_timeout_ns drop the graph. */
scw_status scw_synthesize(scw_plan_t plan, void* out, void* stream);

/* ---- batched sweep (e.g. many wavenumbers of a spectroscopic measurement,
 * Sec. 4.5): n independent items, each with its own orders, layers, grid and
 * wavelength, synthesised by one set of kernels -- one persistent tensor-core
 * contraction over a longest-first task schedule of all items, and batched
 * phase / recompose launches -- replayed as one CUDA graph. All items share the
 * precision; on the tensor-core path they also share the plane-slot count
 * (the largest item's). SCW_FLAG_HOST_IO is not available here.
 *   descs  HOST [n] descriptors (copied); k_split 0 lets the autotuner choose.
 * Set-up work is queued on `stream` and synchronised as in scw_plan. */
scw_status scw_plan_batched(const scw_desc* descs, int n, void* stream, scw_plan_t* out);
/* scw_plan_batched on the legacy default stream. */
scw_status scw_plan_batched_create(const scw_desc* descs, int n, scw_plan_t* out);
/* As scw_plan_set_layers, for item `item` of a batched plan. */
scw_status scw_plan_batched_set_layers(scw_plan_t plan, int item, const void* W, const void* gamma,
                                       const void* alpha, const void* p_inc, const void* p_ref,
                                       const void* p_trn, void* stream);
/* Synthesise every item (Eq. 34 and Eq. 10 per item). The per-item inputs (W,
 * gamma, alpha, p) were bound by scw_plan_batched_set_layers, which converts W
 * into the plan's own layout, so the per-call item table holds the outputs:
 * item i's field is complex64 [3][Fz_i][Fy_i][Fx_i] (or the strided patch its
 * out_ld / out_plane_stride describe). Pass exactly one of
 *   item_table  DEVICE [n] array of DEVICE pointers (8-byte aligned; each
 *               pointer non-NULL and 16-byte aligned -- not checked on the
 *               host, which cannot see them). It is copied on `stream` into the
 *               plan's table, so the call does not synchronise and the table
 *               may be rewritten once that copy has run;
 *   outs        HOST [n] array of DEVICE pointers (checked). The call waits for
 *               the previous call's work on `stream` to have consumed the
 *               plan's pinned staging table before rewriting it.
 * Then one graph launch is queued on `stream`. */
scw_status scw_synthesize_batched(scw_plan_t plan, const void* item_table, void* const* outs, void* stream);
/* Human-readable record of the split choice (model and timed candidates). */
const char* scw_plan_tune_report(scw_plan_t plan);

/* Layer-group pipelining of a single tensor-core plan: the active layers are cut
 * into `groups` contiguous groups; group g's recompose (step c) runs on a
 * second, plan-owned stream while group g+1 is contracted (step b), whose
 * persistent kernel then keeps one CTA per SM so both can share the SMs. The
 * call returns after `stream` has all of it (the second stream joins it).
 * groups = 1 (the default) keeps the serial order. Timed calls
 * (scw_plan_enable_timing) always run serially so their kernel times are
 * separable. Errors: UNSUPPORTED on batched or FP32 plans. */
scw_status scw_plan_set_pipeline(scw_plan_t plan, int groups);

/* Steps (a)+(b) only: the per-plane spectra.
 *   S  DEVICE complex64 [Fz][3][M] (S[z][c][m], Eq. 34 / Eq. 9). */
scw_status scw_spectrum(scw_plan_t plan, void* S, void* stream);

/* Step (c) only: recompose E from caller-given spectra (Eq. 10).
 *   S    DEVICE complex64 [Fz][3][M];  out DEVICE complex64 [3][Fz][Fy][Fx]. */
scw_status scw_recompose(scw_plan_t plan, const void* S, void* out, void* stream);

/* End-to-end through host memory (plan created with SCW_FLAG_HOST_IO): copy
 * W/gamma/alpha/p from HOST buffers of the shapes above, convert, synthesise
 * and copy the field back into HOST `out` [3][Fz][Fy][Fx]. Synchronises the
 * stream before returning. p_* may be NULL without SCW_FLAG_EXTERIOR. */
scw_status scw_synthesize_host(scw_plan_t plan, const void* W, const void* gamma,
                               const void* alpha, const void* p_inc, const void* p_ref,
                               const void* p_trn, void* out, void* stream);

/* ---- fields at arbitrary lateral points (x-z / y-z planes, point sets) -------
 * Eq. 10 evaluated at P given lateral points instead of the Fx x Fy grid:
 *   E_c(x_p, y_p, z_f) = sum_m S_c[m](z_f) exp(2 pi i (u_m x_p / X + v_m y_p / Y))
 * on every z plane f of the plan (z_planes, all illuminations). An x-z plane
 * is the points (x_i, y) for fixed y, a y-z plane (x, y_j) for fixed x; the
 * paper shows fields in all three plane orientations. The sum runs as a dense
 * matrix product over the M orders (no FFT), so points need not lie on a grid,
 * need not be evenly spaced and may lie outside one period (E is periodic).
 *
 * scw_plan_set_points: xy is a HOST double [P][2] array of (x, y), the same
 * length unit as X and Y, finite; 1 <= P <= 2^22 (P = 0 releases the point tables).
 * Builds the plan's table of exp(2 pi i (u x / X + v y / Y)) per (point,
 * order), with the phase reduced in cycles in FP64 (plan-owned: 6 (2M rounded
 * up to 64) bytes per point on tensor-core plans, 8 M bytes on FP32 plans).
 * Synchronises (the device, when it replaces an earlier point set). Single
 * (non-batched) plans only; any number of calls.
 *
 * scw_synthesize_points: out is a DEVICE complex64 [I][3][Fz][P] array
 * (caller-owned, I = illuminations). Runs steps (a) and (b) as scw_synthesize
 * does, then the point product: on tensor-core plans (split-BF16 or FP16 W) a
 * tcgen05 GEMM with split-BF16 operands (hi + lo, three products, FP32
 * accumulation); on FP32 plans a SIMT FP32 GEMM. With timing on, the x-pass
 * slot of scw_kernel_times holds the spectrum operand preparation and the
 * y-pass slot the point product. SCW_ERR_STATE before scw_plan_set_layers or
 * without points; SCW_ERR_UNSUPPORTED on batched plans. */
scw_status scw_plan_set_points(scw_plan_t plan, const double* xy, int n_points);
scw_status scw_synthesize_points(scw_plan_t plan, void* out, void* stream);

/* Scattered points in 3-D: plane is a HOST int [P] array (after scw_plan_set_points) giving each
 * point the index of its z plane in the plan's z_planes, so that point p is evaluated at
 * (x_p, y_p, z_planes[plane[p]]) only. scw_synthesize_points then writes out as DEVICE complex64
 * [I][3][P]: per (point, illumination) one M-term sum of the plane's spectrum (partials of the
 * contraction summed) against the point's row of the point table, on the CUDA cores. NULL returns
 * to every point on every plane. SCW_ERR_STATE without points; INVALID_ARGUMENT for an index
 * outside [0, Fz). Synchronises. */
scw_status scw_plan_set_point_planes(scw_plan_t plan, const int* plane);

/* Synchronise `stream` and read (then clear) the plan's device error word:
 * SCW_OK, SCW_ERR_TIMEOUT (a bounded device wait ran out) or SCW_ERR_CUDA. */
scw_status scw_plan_check(scw_plan_t plan, void* stream);

/* Test hook of SCW_FLAG_DEBUG_BOUNDS plans: lower the extent (in elements) that the checks use
 * for one buffer -- 0 spectra partials, 1 x-pass rows, 2 x twiddles, 3 y twiddles, 4 B operand,
 * 5 gamma, 6 alpha, 7 field, 8 FP32 weights C, 9 FP32 transposed W -- to min(real, elements), or
 * restore the real extent with elements = 0. Accesses the lowered extent rejects are skipped and
 * reported, although they lie inside the real buffer: the checks can be exercised without any
 * access outside an allocation. Drops the graph. SCW_ERR_STATE without the flag. */
scw_status scw_plan_debug_set_extent(scw_plan_t plan, int buffer, unsigned long long elements);

/* Device-side wait limit in nanoseconds for the plan's kernels (default 2 s). */
scw_status scw_plan_set_timeout_ns(scw_plan_t plan, uint64_t ns);

/* Failure injection for tests of the timeout path (on != 0): the first CTA of the
 * tensor-core contraction leaves its first operand stage unfilled, so its bounded
 * waits run out after the plan's timeout; it then lets its issued copies and MMAs
 * land, frees its tensor memory and returns, and the next scw_plan_check reports
 * SCW_ERR_TIMEOUT (the field of that call is invalid). Nothing faults or hangs.
 * UNSUPPORTED for FP32 plans. Drops the graph. */
scw_status scw_plan_inject_stall(scw_plan_t plan, int on);

scw_status scw_plan_get_info(scw_plan_t plan, scw_plan_info* info);

/* Kernel trace of the calls' own launches (graph replay included, where events between kernels
 * would break their programmatic overlap): with tracing on, thread 0 of every CTA stamps the
 * %globaltimer when its work begins (after any wait on the preceding kernel) and when it ends;
 * per slot the earliest begin and the latest end are kept. Slots: 0 phases (a), 1 exterior
 * planes, 2 contraction (b), 3 x-pass and 4 y-pass (c). scw_plan_enable_trace synchronises the
 * device, allocates (on != 0) or frees the 128-byte stamp buffer and drops the graph.
 * scw_plan_get_trace synchronises the device, writes us[2 s] / us[2 s + 1] = begin / end of slot s
 * in microseconds from the earliest begin (-1 for slots no kernel stamped; n_slots entries
 * pairs) and clears the stamps, so each read covers the calls since the previous one.
 * SCW_ERR_STATE when tracing is off. */
scw_status scw_plan_enable_trace(scw_plan_t plan, int on);
scw_status scw_plan_get_trace(scw_plan_t plan, double* us, int n_slots);

/* Per-step kernel durations, measured with CUDA events recorded on the
 * launching stream between the kernels of each scw_synthesize call while
 * timing is enabled (at most 4096 calls are kept). */
typedef struct {
  int calls;             /* synthesize calls averaged                      */
  double phases_ms;      /* step (a) incl. exterior planes, per call       */
  double contract_ms;    /* step (b)                                       */
  double recompose_ms;   /* step (c): both directions and the field stores */
  double xpass_ms;       /* step (c), x direction                          */
  double ypass_ms;       /* step (c), y direction and the field stores     */
  double total_ms;       /* first to last event                            */
} scw_kernel_times;

/* on != 0 starts a new timing window (previous events are dropped). */
scw_status scw_plan_enable_timing(scw_plan_t plan, int on);
/* Synchronises on the recorded events, returns per-call averages and clears them. */
scw_status scw_plan_get_timings(scw_plan_t plan, scw_kernel_times* t);

/* ---- allocation-free recompose ------------------------------------------------
 * The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory -- code that runs inside a host framework's own
 * memory pool, latency-critical loops that must not pay cudaMalloc's implicit
 * device synchronisation, or processes that forbid allocation after start-up.
 * Such callers cannot create a plan (plan creation allocates its workspace), so
 * this call takes the sizes directly and does the recompose step of
 * scw_recompose (x-pass and y-pass) with the same kernels.
 *
 *   S    DEVICE complex64 [Fz][3][U V] spectra (caller-owned input)
 *   out  DEVICE complex64 [3][Fz][Fy][Fx] field (caller-owned output, 16-byte aligned)
 *   U, V, X, Y, Fx, Fy, x0, y0 as in scw_desc; Fz planes.
 *
 * Its scratch is one fixed array of SCW_NOALLOC_SCRATCH_BYTES (8 MiB) compiled
 * into the library as a __device__ variable: every GPU on which the library is
 * loaded holds those 8 MiB until the process exits. A call needs its fold
 * twiddle tables and plane tables,
 *   8 (Fx/8) Ur + 8 (Fy/8) Vr + 12 Fz bytes (each table 256-byte aligned),
 * with Ur, Vr the order counts U, V padded to a multiple of 8 after an offset
 * of at most 7, and returns SCW_ERR_UNSUPPORTED, without launching anything,
 * when that is above the limit. It calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on a device (with that device current) looks up the array's
 * device address with cudaGetSymbolAddress; make that first call before any
 * stream capture. Every call on a device shares the array and it keeps the last
 * call's contents; each call rewrites all of the scratch it reads, so nothing
 * has to be cleared, but calls whose work overlaps on the GPU (different
 * streams, no ordering between them) race on the scratch and corrupt each other. */
#define SCW_NOALLOC_SCRATCH_BYTES (8u << 20)
scw_status scw_recompose_noalloc(int U, int V, double X, double Y, int Fx, int Fy, int Fz, double x0,
                                 double y0, const void* S, void* out, void* stream);

const char* scw_status_string(scw_status s);
const char* scw_last_error(void);
int scw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SCW_H */
