/*
 * degrid.h -- C ABI of the GB300 (sm_103a) 3D degridding library.
 *
 * The operation is the one stated in arXiv:2102.12739, Section
 * "Implementation": given precomputed oversampled gridding convolution
 * functions G_uv (support 8 x 8) and G_w (support 4), a stack of S subgrids
 * of 512 x 512 x 4 regularly sampled visibilities and, for every subgrid, a
 * list of visibility coordinates [u, v, w], compute for every visibility the
 * subgrid point g = [x, y, z] where its footprint starts and the rows of the
 * GCFs to use, then the sum of the 8 x 8 x 4 footprint samples weighted by
 * G_uv times G_w.  The adjoint (gridding) scatters visibilities back with the
 * same weights.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Subgrid stack: C-order [S][ny][nx][nz] complex values (y <-> v,
 *    x <-> u, z <-> w).  Complex values are interleaved (re, im).
 *  - Coordinates: double [N][3] = (u, v, w) in subgrid pixel units with the
 *    origin at element (0, 0, 0).  The lists of consecutive subgrids are
 *    concatenated; vis_offsets [S + 1] (int64, non-decreasing, first 0, last
 *    N) delimits them.
 *  - Snapping (the paper leaves it open; this is the library's definition):
 *    per axis with support W and oversampling O (a power of two),
 *    p = rint(q * O) with ties to even, i = floor(p / O), f = p - i * O,
 *    start = i - W/2 + 1.  A visibility is valid when q is finite,
 *    |q * O| < 2^62 and 0 <= start <= n - W on every axis.  Invalid
 *    visibilities produce 0 (and nothing in the adjoint) and are counted.
 *  - GCF tables: row f, column k holds the kernel value at grid offset
 *    (k - W/2 + 1) - f/O; G_uv is separable, G_uv(a, b) = g_uv[fu][a] *
 *    g_uv[fv][b].
 *  - Device pointers are owned by the caller (a torch tensor's data_ptr() can
 *    be passed directly) and must stay valid until the stream reaches the
 *    work.  Every execute call is asynchronous on the given stream
 *    (cudaStream_t passed as void*, NULL = legacy default stream) and does
 *    not synchronise.
 *  - Argument errors are detected on the host and returned before anything
 *    is enqueued.  Data-dependent conditions (out-of-bounds coordinates,
 *    malformed vis_offsets) are recorded on the device and reported by
 *    degrid_get_status.  No entry point traps or asserts on the device.
 *  - A plan is bound to one device and is not thread-safe: calls on one plan
 *    must not run concurrently from several host threads.
 *  - Calls on one plan share its device scratch (chunk table, claim counter,
 *    status): they must reach the device in order, so issue them on one
 *    stream or order their streams with events.  For work in flight on
 *    several streams at once, use one plan per stream (plans share nothing).
 */
#ifndef DEGRID_H
#define DEGRID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct degrid_plan *degrid_plan_t;

typedef enum {
    DG_OK = 0,
    DG_ERR_ARG = 1,            /* invalid argument (NULL pointer, bad size...) */
    DG_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    DG_ERR_OOM = 3,            /* a device allocation failed */
    DG_ERR_DTYPE = 4,          /* storage type not supported / scale missing */
    DG_ERR_OFFSETS = 5,        /* vis_offsets malformed (found on the device) */
    DG_ERR_UNSUPPORTED = 6,    /* GCF support / subgrid shape not supported */
    DG_ERR_SCRATCH_LIMIT = 7,  /* sizes exceed the fixed scratch of degrid_execute_noalloc */
    DG_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up (found on the device) */
    DG_ERR_BOUNDS = 9          /* an index check of the bounds-checking build failed (on the device) */
} dg_status;

/* Subgrid storage: complex64, or FP16 / BF16 (re, im) pairs with one FP32
 * scale per subgrid (value = code * scale). */
typedef enum {
    DG_C64 = 0,
    DG_C32_F16 = 1,
    DG_C32_BF16 = 2
} dg_dtype;

/* Human-readable name of a status code (static string). */
const char *degrid_status_string(dg_status status);

/* Library version string (static). */
const char *degrid_version(void);

/*
 * Scratch sizing of a plan (host arithmetic only, no GPU needed).  The
 * paper's launch (Eq. 1) needs no scratch; the persistent scheduler here
 * keeps a table of 16-byte work items per plan.  For a GPU with `sm_count`
 * SMs and a plan whose tuned chunk is `plan_chunk` (degrid_plan_set_tuning),
 * a call with n_subgrids subgrids and n_vis visibilities
 *   call_chunk_out  (may be NULL) cuts dense lists into items of this many
 *                   visibilities: plan_chunk, halved (down to 64) while the
 *                   call would give fewer than two items to each of the
 *                   16 * sm_count resident warps;
 *   items_out       (may be NULL) makes the plan reserve this many items
 *                   (16 bytes each): enough for the call itself and for
 *                   every call with at most n_subgrids subgrids and n_vis
 *                   visibilities, whatever chunk those get.  The reserve
 *                   never decreases as n_subgrids or n_vis grow, so after a
 *                   call with the largest sizes no smaller call allocates.
 * Returns DG_ERR_ARG for sm_count < 1, a plan_chunk that is not a multiple
 * of 32 in [32, 65536], or negative sizes.
 */
dg_status degrid_schedule_reserve(int sm_count, int plan_chunk, int n_subgrids, int64_t n_vis,
                                  int *call_chunk_out, int64_t *items_out);

/*
 * Create a plan (Section "Implementation": the precomputed oversampled GCFs
 * and the 512 x 512 x 4 subgrid shape are the fixed inputs of the method).
 *   out            receives the plan handle (set to NULL on failure)
 *   nx, ny, nz     subgrid extent; layout [S][ny][nx][nz]; nz >= w_support,
 *                  ny * nx * nz < 2^31, max(nx, ny) * uv_oversample <= 2^31
 *                  and nz * w_oversample <= 2^31 (else DG_ERR_UNSUPPORTED)
 *   g_uv           HOST double [uv_oversample][uv_support], copied (and
 *                  rounded to FP32) to the device; the caller keeps it
 *   uv_support     must be 8 (the paper's 8 x 8 footprint)
 *   uv_oversample  power of two, 1 .. 2^20
 *   g_w            HOST double [w_oversample][w_support], copied likewise
 *   w_support      must be 4
 *   w_oversample   power of two, 1 .. 2^20
 *   dtype          storage type of the subgrids passed to degrid_execute
 *   device         CUDA device ordinal; it is made current for the call
 * Returns DG_OK, DG_ERR_ARG, DG_ERR_UNSUPPORTED, DG_ERR_OOM or DG_ERR_CUDA.
 */
dg_status degrid_plan_create(degrid_plan_t *out, int nx, int ny, int nz,
                             const double *g_uv, int uv_support, int uv_oversample,
                             const double *g_w, int w_support, int w_oversample,
                             dg_dtype dtype, int device);

/*
 * Create a plan with a non-separable G_uv (the paper states G_uv as a kernel
 * of support 8 x 8, Section "Implementation"; degrid_plan_create takes the
 * separable special case g(a) g(b) at high oversampling).
 *   g_uv2          HOST double [uv_oversample][uv_oversample][8][8], indexed
 *                  [fv][fu][b][a]: block (fv, fu) holds the weight of
 *                  footprint point (row b along v, column a along u) for
 *                  oversampled offsets fv and fu; copied (rounded to FP32)
 *   uv_oversample  power of two, 1 .. DG_TABLE2D_MAX_OVERSAMPLE (the FP32
 *                  table, uv_oversample^2 * 256 bytes, stays L2-resident)
 * and the other arguments as for degrid_plan_create (support 8 implied).
 * degrid_execute (all storage types, compensated or not) and
 * grid_adjoint_execute use the 2D table; the direct summing arm is not used.
 */
#define DG_TABLE2D_MAX_OVERSAMPLE 256
dg_status degrid_plan_create_2d(degrid_plan_t *out, int nx, int ny, int nz, const double *g_uv2,
                                int uv_oversample, const double *g_w, int w_support,
                                int w_oversample, dg_dtype dtype, int device);

/* Release the plan and every device buffer it owns.  Synchronises the
 * plan's device first.  NULL is ignored. */
void degrid_plan_destroy(degrid_plan_t plan);

/*
 * Tuning knobs of the persistent degridding / gridding kernels (the paper
 * tunes N_b, the visibilities per thread block, by hand; Section "Results").
 *   chunk            visibilities per work item claimed by one warp
 *                    (multiple of 32, 32 .. 65536); a work item never
 *                    straddles two subgrids.  Lists of fewer than
 *                    64 * chunk visibilities (sparse: few visibilities
 *                    share a footprint) are cut into items of 64 instead
 *                    and claimed before the others, so that no costly
 *                    item is left for the end of a call (chunk > 64;
 *                    results do not depend on it).  A call too small for
 *                    two items per resident warp halves its chunk, down to
 *                    64, so that it still spreads over the GPU.  Every item
 *                    is one atomic claim on a single device-wide counter:
 *                    items of fewer than 64 visibilities (one pipeline step) make
 *                    every step a claim and the counter then bounds the
 *                    call (gridding measured 18x slower at 32 than at
 *                    256); 128 .. 1024 is the useful range, the one the
 *                    autotuner searches
 *   warps_per_block  warps per CTA (1 .. 32)
 *   blocks_per_sm    resident CTAs per SM for the persistent grid
 *                    (0 = as many as the occupancy calculator allows)
 * Any argument <= 0 keeps the current value, except blocks_per_sm where 0
 * selects the occupancy maximum and < 0 keeps the current value.
 * Returns DG_OK or DG_ERR_ARG.
 */
dg_status degrid_plan_set_tuning(degrid_plan_t plan, int chunk, int warps_per_block,
                                 int blocks_per_sm);

/*
 * Compensated reduction (the precision pattern of the target: FP32
 * accumulation with compensated summation of the partial sums that lanes
 * exchange).  With enabled = 1, every addition of the cross-lane reduction of
 * degrid_execute is an error-free TwoSum (Knuth) and the rounding errors are
 * added back at the end, so the combination of the four lane partials of a
 * visibility is exact before one final rounding; the per-lane FMA chains are
 * unchanged.  enabled = 0 (the default) adds the partials plainly.  Both
 * forms are deterministic.  Returns DG_OK, or DG_ERR_ARG for a NULL plan or
 * a value other than 0 / 1.  Not used by grid_adjoint_execute.
 */
dg_status degrid_plan_set_compensated(degrid_plan_t plan, int enabled);
dg_status degrid_plan_get_compensated(degrid_plan_t plan, int *enabled);

/*
 * Summing arm for short runs (the paper's per-visibility kernels D1/D2 next
 * to the footprint-reuse path, Section "Implementation").  degrid_execute
 * works on halves of 32 consecutive visibilities.  A half whose visibilities
 * share one footprint and w row reuses the cached footprint sum M; any other
 * half with at least min_runs runs of equal (footprint, w row) is summed
 * directly, every visibility from its own 8 x 8 x 4 footprint (no cache
 * rebuilds), and halves with fewer runs rebuild M per run.  Both arms do the
 * same arithmetic in the same order, so the results are bitwise identical;
 * only the speed differs: the direct arm wins on lists whose footprints
 * overlap but change often (w rows changing every few visibilities) and
 * loses on footprints scattered over the subgrid.  min_runs: 1 ..
 * DG_DIRECT_RUNS_NEVER (33: never, the default; a plan with the arm enabled
 * launches another instance of the kernel).  DG_DIRECT_RUNS_SHORT is the
 * setting the autotuner tries.  Returns DG_OK or DG_ERR_ARG.
 */
#define DG_DIRECT_RUNS_NEVER 33
#define DG_DIRECT_RUNS_DEFAULT DG_DIRECT_RUNS_NEVER
#define DG_DIRECT_RUNS_SHORT 9
dg_status degrid_plan_set_direct_runs(degrid_plan_t plan, int min_runs);
dg_status degrid_plan_get_direct_runs(degrid_plan_t plan, int *min_runs);

/*
 * Gather arm for sparse coverage (lists whose consecutive visibilities
 * rarely share a footprint: the short-list regime of the paper's kernels
 * D2/D4, Section "Results").  With enabled = 1, degrid_execute streams every
 * visibility's own 8 x 8 x 4 footprint into shared memory with asynchronous
 * copies, several footprints in flight per warp, instead of caching the
 * footprint sum M per run; a separate kernel with one CTA per SM (12 warps
 * for complex64, 22 for FP16/BF16), so the warps_per_block and
 * blocks_per_sm of the tuning do not apply to it (the chunk size does).
 * Same arithmetic in the same order as the footprint-cache path: results
 * are bitwise identical; the compensated setting applies.  Only the speed
 * differs: it wins when footprints are scattered and loses on dense lists,
 * where one cached M serves hundreds of visibilities.  The setting also
 * switches grid_adjoint_execute (output stack 16-byte aligned) to its
 * counterpart for scattered coverage: each visibility's 8 x 8 x 4
 * contribution is written to shared memory and added to the stack by one
 * tensor reduce-add of the copy engine, instead of the run accumulation
 * with atomic adds at run ends (FP32 additions in another order: the last
 * bits differ).  Needs nz = 4 and a separable G_uv table: enabling it on another
 * plan returns DG_ERR_UNSUPPORTED.  Calls whose stack has more than
 * 2^31 - 1 rows in all (n_subgrids * ny) take the footprint-cache kernels
 * whatever the setting (the copy engine's row coordinate is 32-bit).
 * Returns DG_OK, DG_ERR_ARG (enabled not 0 / 1) or DG_ERR_UNSUPPORTED.
 */
dg_status degrid_plan_set_gather(degrid_plan_t plan, int enabled);
dg_status degrid_plan_get_gather(degrid_plan_t plan, int *enabled);

/* Read back the current tuning (any pointer may be NULL). */
dg_status degrid_plan_get_tuning(degrid_plan_t plan, int *chunk, int *warps_per_block,
                                 int *blocks_per_sm);

/*
 * Kernel timing (profiling aid, not in the paper).  degrid_plan_enable_timing
 * with n_slots > 0 creates n_slots CUDA event pairs; from then on every
 * degrid_execute / grid_adjoint_execute records one pair on its stream around
 * its main (persistent) kernel only, excluding the small scheduling
 * kernels, cycling through the slots.  n_slots = 0 disables timing and frees
 * the events.  Disable timing before capturing calls into a CUDA graph.
 *
 * degrid_plan_kernel_times_ms synchronises on the newest pair and writes the
 * durations (milliseconds) of the most recent min(capacity, launches,
 * n_slots) timed launches to ms_out, oldest first, and their number to
 * *count.  Timing another launch resets nothing: slots are reused in turn.
 * Both return DG_OK, DG_ERR_ARG or DG_ERR_CUDA.
 */
dg_status degrid_plan_enable_timing(degrid_plan_t plan, int n_slots);
dg_status degrid_plan_kernel_times_ms(degrid_plan_t plan, float *ms_out, int capacity,
                                      int *count);

/*
 * FP32 arithmetic peak of `device`, measured (the denominator of the
 * degridding roofline: the footprint sum of Section "Implementation" is
 * bound by FP32 fused multiply-adds).  Runs 8 CTAs of 256 threads per SM,
 * each thread 16 independent FMA chains, as packed two-wide FFMA2
 * (packed != 0, the form the degridding kernel issues) or scalar FFMA, and
 * times 5 launches of about 4 ms after a warm-up one with CUDA events on a
 * stream of its own.  *tflops receives the best launch's 2 flop per lane FMA
 * divided by its duration, in TFLOP/s.  Synchronous; allocates and frees
 * 1.2 MB of device memory.  Returns DG_OK, DG_ERR_ARG (tflops NULL or
 * device < 0), DG_ERR_OOM or DG_ERR_CUDA.
 */
dg_status degrid_measure_fp32_peak(int device, int packed, double *tflops);

/*
 * L2-to-SM read bandwidth of `device`, measured (the no-reuse gather bound:
 * without footprint reuse every visibility reads its own 8 x 8 x 4
 * footprint, 2 KB in complex64 or 1 KB in FP16/BF16, from L2).  Runs 8 CTAs
 * of 256 threads per SM that read an L2-resident buffer (8 x 16 bytes per
 * thread, 39.8 MB on 152 SMs) 1000 times with L1-bypassing 16-byte loads,
 * and times 5 launches after a warm-up one with CUDA events on a stream of
 * its own.  *gbs receives the bytes read by the best launch divided by its
 * duration, in GB/s (1e9 bytes).  Synchronous; allocates and frees the
 * buffer.  Returns DG_OK, DG_ERR_ARG (gbs NULL or device < 0), DG_ERR_OOM or
 * DG_ERR_CUDA.
 */
dg_status degrid_measure_l2_read_bw(int device, double *gbs);

/*
 * The rate, in GB/s of added data, at which the copy engines apply tensor
 * reduce-adds of 2 KB footprint tiles (8 rows x 256 bytes of FP32 pairs at
 * footprint positions) into an L2-resident stack, one stream of them per
 * warp of a CTA of 16 warps on every SM: the bound of the gridding kernel
 * for scattered coverage (no counterpart in the paper).  Synchronous; makes
 * `device` current for the call.  Returns DG_OK, DG_ERR_ARG, DG_ERR_OOM or
 * DG_ERR_CUDA.
 */
dg_status degrid_measure_l2_reduce_bw(int device, double *gbs);

/*
 * Degridding (Section "Implementation", the weighted footprint sum):
 *   vis_out[i] = sum_{b<8} sum_{a<8} sum_{c<4} g_uv[fv][b] g_uv[fu][a]
 *                g_w[fw][c] * sub[s][y0+b][x0+a][z0+c]
 * for every visibility i of subgrid s, in the order of uvw.
 *   stream         cudaStream_t (as void*), NULL = legacy default stream
 *   n_subgrids     S >= 0
 *   subgrids       DEVICE, S * ny * nx * nz complex values in the plan's
 *                  storage type (8 bytes each for DG_C64, 4 bytes otherwise);
 *                  16-byte aligned
 *   subgrid_scale  DEVICE float [S]; required for DG_C32_F16 / DG_C32_BF16,
 *                  ignored (may be NULL) for DG_C64
 *   uvw            DEVICE double [n_vis][3], 8-byte aligned
 *   vis_offsets    DEVICE int64 [S + 1]
 *   n_vis          N >= 0 (must equal vis_offsets[S])
 *   vis_out        DEVICE float [n_vis][2] (complex64), 8-byte aligned;
 *                  every element is written
 * Accumulation is FP32; the coordinate step is exact integer arithmetic on
 * the FP64 coordinates.  Malformed vis_offsets are flagged for
 * degrid_get_status; subgrids with a negative count are skipped.
 * The plan's scratch grows on the first call with a larger S or N (see
 * degrid_schedule_reserve: what a call reserves covers every call with
 * smaller S and N); call once with the largest sizes before capturing calls
 * in a CUDA graph.
 */
dg_status degrid_execute(degrid_plan_t plan, void *stream, int n_subgrids,
                         const void *subgrids, const float *subgrid_scale,
                         const double *uvw, const int64_t *vis_offsets, int64_t n_vis,
                         float *vis_out);

/*
 * degrid_execute with the inputs and the output in HOST memory (no
 * counterpart in the paper, which starts from data on the GPU), in one of two
 * ways:
 *  - in place, when subgrids, uvw and vis_out are page-locked (pinned: mapped
 *    into the GPU's address space) and the plan allows it (the default, see
 *    degrid_plan_set_host_direct) and does not use the gather kernel: the
 *    kernel reads the coordinates and the footprint rows it needs directly
 *    from host memory over the host link and writes the visibilities there;
 *    only vis_offsets (and the scales, if not pinned) are copied.  A dense
 *    list reads a small part of its subgrid, so this moves far fewer bytes
 *    than copying the stack;
 *  - otherwise by copies: the subgrids, coordinates and offsets go to the
 *    device and the visibilities come back, overlapping the copies with the
 *    sums: the stack is processed in groups of consecutive subgrids (about
 *    64 MB of subgrid data each) through two device slots, with the copy-in
 *    of one group, the sums of the previous one and the copy-out of the one
 *    before that on three streams of the plan.  Groups without visibilities
 *    are not copied.
 * Both give the results of degrid_execute bit for bit.  The call returns when
 * vis_out is complete (synchronous; the plan's streams are not the caller's).
 *   subgrids, subgrid_scale, uvw, vis_offsets, vis_out   HOST pointers, the
 *                  layouts of degrid_execute; pinned memory gives the in-place
 *                  form (or full copy bandwidth and overlap), pageable memory
 *                  works by copies at lower speed
 * vis_offsets is checked on the host: DG_ERR_OFFSETS if vis_offsets[0] != 0,
 * vis_offsets[S] != n_vis or it decreases.  The first call allocates the
 * plan's streams and two staging slots (grown when a later call needs more);
 * degrid_plan_destroy frees them.  Invalid visibilities are counted as for
 * degrid_execute (read them with degrid_get_status).  Returns DG_OK,
 * DG_ERR_ARG, DG_ERR_DTYPE, DG_ERR_OFFSETS, DG_ERR_OOM or DG_ERR_CUDA.
 */
dg_status degrid_execute_host(degrid_plan_t plan, int n_subgrids, const void *subgrids,
                              const float *subgrid_scale, const double *uvw,
                              const int64_t *vis_offsets, int64_t n_vis, float *vis_out);

/*
 * Whether degrid_execute_host may read page-locked host inputs in place
 * (enabled = 1, the default) or always copies them (0).  Returns DG_OK or
 * DG_ERR_ARG.
 */
dg_status degrid_plan_set_host_direct(degrid_plan_t plan, int enabled);
dg_status degrid_plan_get_host_direct(degrid_plan_t plan, int *enabled);

/*
 * Adjoint of degrid_execute (gridding): for every visibility i of subgrid s
 *   sub_out[s][y0+b][x0+a][z0+c] += g_uv[fv][b] g_uv[fu][a] g_w[fw][c] * vis_in[i]
 * (real weights, so the adjoint needs no conjugation).  sub_out is complex64
 * [S][ny][nx][nz] on the DEVICE, zeroed first unless accumulate != 0.
 * FP32 atomic accumulation (16-byte vector reductions when nz = 4 and
 * sub_out is 16-byte aligned, float2 atomics otherwise): the summation
 * order, and so the last bits, are not deterministic.  Other arguments as
 * for degrid_execute.  With a plan made
 * by degrid_plan_create_2d the weights are G[fv][fu][b][a] g_w[fw][c].
 */
dg_status grid_adjoint_execute(degrid_plan_t plan, void *stream, int n_subgrids,
                               const double *uvw, const int64_t *vis_offsets,
                               int64_t n_vis, const float *vis_in, float *sub_out,
                               int accumulate);

/*
 * Coordinate step alone (Section "Implementation": the start point g and the
 * GCF locations of every visibility), as computed inside degrid_execute:
 * coords_out DEVICE int32 [n_vis][6] = (x0, y0, z0, fu, fv, fw), all six -1
 * for an invalid visibility (which is also counted for degrid_get_status).
 */
dg_status degrid_coords_execute(degrid_plan_t plan, void *stream, const double *uvw,
                                int64_t n_vis, int32_t *coords_out);

/*
 * Convert complex64 subgrids to the reduced-precision storage used by
 * DG_C32_F16 / DG_C32_BF16: scale[s] = max over subgrid s of
 * max(|re|, |im|); code = round-to-nearest-even(component / scale) in the
 * target format (FP32 division); an all-zero subgrid gets scale 0 and zero
 * codes.  Not part of the paper (its subgrids are given); provided so that
 * callers can produce the storage the kernels read.
 *   dtype        DG_C32_F16 or DG_C32_BF16
 *   elems        complex elements per subgrid (ny * nx * nz)
 *   in           DEVICE float [S][elems][2]
 *   codes_out    DEVICE uint16 [S][elems][2]
 *   scale_out    DEVICE float [S]
 */
dg_status degrid_pack_subgrids(void *stream, dg_dtype dtype, int n_subgrids, int64_t elems,
                               const float *in, void *codes_out, float *scale_out);

/*
 * Read and clear the device-side status of the plan: synchronises `stream`,
 * stores the number of invalid visibilities seen since the last call in
 * *n_invalid (may be NULL) and returns DG_ERR_TIMEOUT if a bounded wait of
 * a kernel gave up (the gather kernel's waits on its copies; the results of
 * that call are incomplete), else DG_ERR_BOUNDS if the library was built
 * with DEGRID_BOUNDS_CHECK and an index the coordinate step produced fell
 * outside its buffer (that visibility was skipped), else DG_ERR_OFFSETS if a
 * call saw malformed vis_offsets, else DG_OK (or DG_ERR_CUDA).
 */
dg_status degrid_get_status(degrid_plan_t plan, void *stream, int64_t *n_invalid);

/*
 * Degridding without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc once they
 * are running, such as real-time pipelines that must not enter the CUDA
 * allocator after start-up (allocation and release can synchronise the
 * device and stall every other stream) and hosts whose device-memory budget
 * is owned entirely by another allocator.
 *
 * It computes the same visibilities as degrid_execute, but takes no plan:
 *   g_uv, g_w      DEVICE float tables [uv_oversample][8] and [w_oversample][4]
 *                  (the FP32 values degrid_plan_create would store)
 *   nx, ny, nz,    as for degrid_plan_create (supports 8 and 4 implied;
 *                  a shape outside its limits gives DG_ERR_ARG here)
 *   uv_oversample, w_oversample, dtype
 *   status_out     DEVICE unsigned long long [2] or NULL: receives the number
 *                  of invalid visibilities and error flags (bit 0: malformed
 *                  vis_offsets) of this call; zeroed by the call
 * and the remaining arguments as for degrid_execute.  Every call is
 * asynchronous on `stream` and uses the device that is current.
 *
 * All scratch comes from one fixed array of DG_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  Calls with
 * uv_oversample > DG_NOALLOC_MAX_UV_OVERSAMPLE, w_oversample >
 * DG_NOALLOC_MAX_W_OVERSAMPLE, n_subgrids > DG_NOALLOC_MAX_SUBGRIDS or
 * n_vis > DG_NOALLOC_MAX_VIS are rejected with DG_ERR_SCRATCH_LIMIT before
 * anything is enqueued.  The array is shared by all calls on a device and
 * keeps what the previous call left, so calls whose work overlaps on the GPU
 * (different streams, or different host threads) race with each other and
 * must be serialised by the caller.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.
 */
#define DG_NOALLOC_SCRATCH_BYTES (1024u * 1024u)
#define DG_NOALLOC_MAX_UV_OVERSAMPLE (1 << 20)
#define DG_NOALLOC_MAX_W_OVERSAMPLE 512
#define DG_NOALLOC_MAX_SUBGRIDS 1024
#define DG_NOALLOC_MAX_VIS (1 << 25)
dg_status degrid_execute_noalloc(void *stream, int nx, int ny, int nz,
                                 const float *g_uv, int uv_oversample,
                                 const float *g_w, int w_oversample, dg_dtype dtype,
                                 int n_subgrids, const void *subgrids,
                                 const float *subgrid_scale, const double *uvw,
                                 const int64_t *vis_offsets, int64_t n_vis,
                                 float *vis_out, unsigned long long *status_out);

/*
 * The subgrid stack itself: the step upstream of degridding.  The paper
 * takes the stack as "pre-computed grid data" of the improved w-stacking
 * method (Introduction) and does not describe it; following improved
 * w-stacking (Ye, Gull, Tan & Nikolic 2020), the grid at a w-plane is the
 * Fourier transform of the corrected sky image times the plane's w-phase
 * screen.  For an N x N image I (row b <-> m, column a <-> l, direction
 * cosines l_a = (a - N/2) theta / N, m_b likewise) and a real image-plane
 * correction T, subgrid s is
 *   G[s][y][x][c] = sum_{b,a} I[b][a] T[b][a]
 *       exp(-2 pi i ((x - N/2 + u0_s)(a - N/2) / N + (y - N/2 + v0_s)(b - N/2) / N
 *                     + (w0_s + c dw_s)(n_ab - 1))),   n_ab = sqrt(1 - l_a^2 - m_b^2),
 * for cells x, y < N and w-planes c < nz (pixels with l^2 + m^2 >= 1 add
 * nothing): the uv cells (x - N/2 + u0_s, y - N/2 + v0_s) / theta
 * wavelengths at w = w0_s + c dw_s, laid out [S][N][N][nz] as degrid_execute
 * reads them (DG_C64).
 *
 * subgrid_predict_plan_create
 *   n                  image and subgrid side N: even, >= 8, N * N * nz < 2^31
 *   nz                 w-planes per subgrid, 1 .. 64 (4 for the paper's stack)
 *   subgrids_per_pass  subgrids transformed together (1 .. 4096); the plan
 *                      holds a work buffer of subgrids_per_pass * nz * N * N
 *                      complex64 and a batched 2D FFT plan (cuFFT)
 *   device             CUDA device ordinal
 * Returns DG_OK, DG_ERR_ARG, DG_ERR_OOM or DG_ERR_CUDA.
 *
 * subgrid_predict_execute (asynchronous on `stream`; no allocation)
 *   theta         image width in direction cosines (> 0, finite)
 *   image         DEVICE complex64 [N][N], 8-byte aligned
 *   taper         DEVICE float [N][N] (the gridding correction T), or NULL for 1
 *   n_subgrids    S >= 0
 *   uv_offsets    DEVICE int32 [S][2]: (u0_s, v0_s) integer cell offsets
 *   w_planes      DEVICE double [S][2]: (w0_s, dw_s) in wavelengths
 *   subgrids_out  DEVICE complex64 [S][N][N][nz], every element written
 * Returns DG_OK, DG_ERR_ARG (NULL or misaligned pointers, bad theta) or
 * DG_ERR_CUDA.  Arithmetic: FP32; the w-phase w (n - 1) is reduced to a
 * fraction of a turn in double-float arithmetic (exact to about 3e-8 turns
 * while |w (n - 1)| < 2^22 turns) before its sine and cosine.
 */
typedef struct subgrid_predict_plan *subgrid_predict_plan_t;
dg_status subgrid_predict_plan_create(subgrid_predict_plan_t *out, int n, int nz, int subgrids_per_pass,
                                      int device);
dg_status subgrid_predict_execute(subgrid_predict_plan_t plan, void *stream, double theta,
                                  const float *image, const float *taper, int n_subgrids,
                                  const int32_t *uv_offsets, const double *w_planes,
                                  float *subgrids_out);
void subgrid_predict_plan_destroy(subgrid_predict_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* DEGRID_H */
