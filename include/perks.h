/*
 * perks.h -- C ABI of the GB300 (sm_103a) persistent-kernel solver library.
 *
 * The library implements the PERKS execution model of arXiv 2204.02064
 * ("PERKS: a Locality-Optimized Execution Model for Iterative Memory-bound
 * GPU Applications", Sec. 3-4): the time/iteration loop of an iterative
 * memory-bound solver runs inside ONE cooperative kernel launch with a
 * device-wide barrier per step, and every thread block keeps its tile of the
 * state in registers and shared memory between steps, so that only halos and
 * the uncached remainder travel through L2/HBM.
 *
 * Two solvers are exposed:
 *   - Jacobi stencils (Eq. iterativeStencil, Sec. 2.2.1; Sec. 4.2):
 *     y(c) = sum_o w_o x(c + o) over 2-D / 3-D grids with a fixed Dirichlet
 *     boundary, run for N steps;
 *   - conjugate gradient (Sec. 2.2.2; Sec. 4.3) on a CSR matrix, with the
 *     merge-path SpMV, dot products and axpys fused into the same persistent
 *     loop, solved to a relative residual tolerance.
 *
 * Conventions (all entry points):
 *   - Return value: perks_status, 0 on success, a negative PERKS_ERR_* code on
 *     failure.  No exception, abort or exit crosses the ABI.  A human-readable
 *     message for the last failure is kept per context (perks_last_error).
 *   - Pointers: "host" pointers are ordinary CPU memory (pinned or pageable);
 *     "device" pointers are CUDA global memory of the context's device (for
 *     example torch.Tensor.data_ptr()).  Each call that takes a buffer says
 *     which, or takes an on_device flag.
 *   - Ownership: the library copies every input into device memory it owns
 *     and frees it in the matching *_destroy.  Caller buffers passed to a
 *     stream-ordered call must stay valid until that stream reaches the call.
 *   - Streams: `perks_stream` is a cudaStream_t (NULL = legacy default
 *     stream).  Calls are stream-ordered; run/solve return before the GPU
 *     finishes unless they are asked for statistics, in which case they
 *     synchronize the stream and report device-side errors.
 *   - Threading: a context and the objects made from it must not be used by
 *     two host threads at the same time.
 *   - Layout: grids are row-major with x fastest: element (x, y, z) of an
 *     nx*ny*nz grid is at index x + nx*(y + ny*z); a 2-D grid is nx*ny.
 */
#ifndef PERKS_H
#define PERKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int perks_status;

#define PERKS_OK 0
#define PERKS_ERR_INVALID_ARG (-1)       /* a NULL, size or descriptor error */
#define PERKS_ERR_UNSUPPORTED (-2)       /* valid request the library does not implement */
#define PERKS_ERR_OUT_OF_MEMORY (-3)     /* a device allocation failed */
#define PERKS_ERR_LAUNCH_TOO_LARGE (-4)  /* grid not co-resident (Sec. 4.4.1: no oversubscription) */
#define PERKS_ERR_CUDA (-5)              /* any other CUDA runtime error */
#define PERKS_ERR_BARRIER_TIMEOUT (-6)   /* a grid barrier wait ran past its limit */
#define PERKS_ERR_NOT_CONVERGED (-7)     /* CG hit max_iter above tolerance */
#define PERKS_ERR_BREAKDOWN (-8)         /* CG: <p, Ap> <= 0 or not finite */

typedef struct perks_context perks_context;
typedef struct perks_stencil perks_stencil;
typedef struct perks_op perks_op;
typedef void *perks_stream; /* cudaStream_t */

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (queries SM count, shared memory
 * and co-residency limits).  *out receives the handle; free it with
 * perks_context_destroy.  Errors: INVALID_ARG (out NULL or bad device),
 * CUDA. */
perks_status perks_context_create(int device, perks_context **out);
/* Frees the context.  Objects created on it may still be destroyed
 * afterwards (their destroy calls do not touch the context); every other
 * call on them needs the context alive. */
perks_status perks_context_destroy(perks_context *ctx);

/* Message of the last failed call on this context (or on an object made
 * from it).  Owned by the context; valid until its next call.  Never NULL. */
const char *perks_last_error(const perks_context *ctx);

/* Limit, in nanoseconds, of every grid-barrier wait inside persistent
 * kernels launched from this context (default 2e9).  A wait that runs past
 * it makes the kernel stop all blocks cleanly and the run/solve report
 * BARRIER_TIMEOUT; 0 makes every wait give up at once (used to test the
 * error path).  Errors: INVALID_ARG (ctx NULL or limit < 0). */
perks_status perks_context_set_barrier_timeout(perks_context *ctx, int64_t limit_ns);

/* Grid-synchronisation cost (a measurement aid): times one cooperative
 * launch of `blocks` x `threads` that runs `iterations` of the persistent
 * kernels' grid barrier and nothing else (after one warm-up launch), and
 * returns the mean microseconds per barrier.  Errors: INVALID_ARG,
 * LAUNCH_TOO_LARGE (blocks not co-resident), BARRIER_TIMEOUT, CUDA. */
perks_status perks_barrier_benchmark(perks_context *ctx, int32_t blocks, int32_t threads,
                                     int32_t iterations, double *us_per_barrier);

/* FP64 pipe throughput (a measurement aid, not in the paper): times one
 * launch (after a warm-up launch) of 4 blocks of 256 threads per SM, each
 * thread running eight independent chains of `iterations` fp64 fused
 * multiply-adds, and returns the rate in TFLOP/s (2 FLOP per FMA).  The
 * ceiling of stencils whose fp64 arithmetic, not memory, bounds a step.
 * Errors: INVALID_ARG, CUDA. */
perks_status perks_fp64_fma_benchmark(perks_context *ctx, int32_t iterations, double *tflops);

/* Random-gather throughput (a measurement aid, not in the paper): times one
 * launch (after a warm-up launch that also brings the vector into L2) of 4
 * blocks of 256 threads per SM, each thread issuing `iterations` x 8
 * independent cache-global loads of elem_bytes (4 or 8) at pseudo-random
 * positions of a vector of 2^log2_elems elements (10..28), and returns the
 * loads per second: the ceiling of an SpMV whose column indices are
 * scattered over a vector that L2 holds (one 32-byte sector per gathered
 * value).  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
perks_status perks_gather_benchmark(perks_context *ctx, int32_t log2_elems, int32_t elem_bytes,
                                    int32_t iterations, double *gathers_per_s);

/* Device facts used by planners and reports: SM count, opt-in shared memory
 * per block (bytes), L2 size (bytes).  Any out pointer may be NULL. */
perks_status perks_context_info(const perks_context *ctx, int32_t *sm_count,
                                int32_t *smem_per_block, int64_t *l2_bytes);

/* ------------------------------------------------------------------------ */
/* Jacobi stencils: Eq. (iterativeStencil), Sec. 2.2.1; PERKS port, Sec. 4.2 */
/* ------------------------------------------------------------------------ */

#define PERKS_MAX_POINTS 125

enum { PERKS_F64 = 0, PERKS_F32 = 1, PERKS_BF16 = 2 };
enum { PERKS_PERSISTENT = 0, PERKS_PER_STEP = 1 };

typedef struct {
    int32_t ndim;                       /* 2 or 3 */
    int64_t nx, ny, nz;                 /* interior extents; nz must be 1 when ndim == 2 */
    int32_t radius;                     /* 1..4: ghost ring width, max |offset|; the persistent
                                           kernels cover the compiled shapes (radius 1 and 2, and
                                           the 2-D stars of radius 3 and 4 with nx a multiple of
                                           16 bytes, those without on-chip caches); other shapes
                                           run the per-step variant only */
    int32_t npts;                       /* number of (offset, weight) pairs, 1..PERKS_MAX_POINTS */
    int32_t offsets[3 * PERKS_MAX_POINTS]; /* (dx, dy, dz) per point; dz = 0 in 2-D */
    double weights[PERKS_MAX_POINTS];   /* w_o, applied in the storage dtype's accumulator */
    int32_t dtype;                      /* PERKS_F64, PERKS_F32 (fp32 accumulate), PERKS_BF16 (fp32 accumulate) */
    double boundary;                    /* Dirichlet value of every cell outside the interior */
} perks_stencil_desc;

/* Optional plan override for the persistent kernel (all zero = automatic).
 * Tile counts split each axis into nearly equal parts, one tile per block. */
typedef struct {
    int32_t tiles_x, tiles_y, tiles_z;
    int32_t smem_cache_planes;          /* -1: as many as fit; >= 0: at most this many */
    int32_t reg_cache;                  /* plane streaming: 0 no register cache, 1 the compiled
                                           register depth; resident tile: rows per thread
                                           (1 or 2, 0 = automatic) */
    int32_t reserved[4];                /* reserved[0] = 1: one-cell-per-thread kernel instead of
                                           the 16-byte-vector kernel; reserved[1] = planes per
                                           block barrier of the vector kernel (2 or 4, 0 =
                                           automatic); reserved[2] = kernel body
                                           (PERKS_KERNEL_AUTO / _RESIDENT / _STREAMING; AUTO in a
                                           plan means STREAMING, AUTO with no plan picks the
                                           resident tile when every tile fits in shared memory);
                                           reserved[3] = threads per block (0 = automatic):
                                           256 or 512 for the resident tile kernel; 256 picks the
                                           plane-streaming kernel's two-blocks-per-SM
                                           instantiations where they exist (fp64 3d7pt,
                                           cache-free body) */
    int32_t balanced;                   /* plane streaming with no caches (reg_cache = 0,
                                           smem_cache_planes = 0): 1 = the tiles_x x tiles_y
                                           tile columns are laid end to end (each column all
                                           its planes in z) and cut into equal contiguous
                                           shares, one per co-resident block, so every block
                                           gets the same number of planes whatever the block
                                           count (a share may end one column and start the
                                           next); tiles_z is ignored.  0 = one tile per block */
} perks_stencil_plan;

/* What a run did; filled by perks_stencil_run when asked. */
typedef struct {
    int64_t steps;
    int32_t variant;                    /* PERKS_PERSISTENT or PERKS_PER_STEP */
    int32_t grid_blocks, threads_per_block;
    int32_t tiles_x, tiles_y, tiles_z;  /* internal orientation: 2-D y maps to z */
    int32_t reg_cache_planes, smem_cache_planes;  /* resident tile: rows per thread, planes per tile */
    int32_t prefetch_planes;
    int64_t smem_bytes_per_block;
    int64_t cells;                      /* interior cells */
    int64_t cached_cells;               /* cells held on chip between steps (D_cache) */
    int64_t halo_cells_per_step;        /* halo cells written + read per step (H) */
    double algorithmic_bytes;           /* S (2 N D_uncache + 2 D_cache) + S N H for the whole run */
    int32_t kernel;                     /* PERKS_KERNEL_*: which kernel body runs */
    int32_t planes_per_sync;            /* resident tile: planes a thread computes between two block
                                           barriers; plane streaming: planes per block barrier */
} perks_run_stats;

/* Kernel bodies of a stencil run (perks_run_stats.kernel, perks_stencil_plan.reserved[2]). */
enum {
    PERKS_KERNEL_AUTO = 0,       /* plan field only: choose automatically */
    PERKS_KERNEL_RESIDENT = 1,   /* resident tile: every block keeps its whole tile in shared memory
                                    for all steps (radius-1 stars: 2d5pt, 3d7pt) */
    PERKS_KERNEL_STREAMING = 2,  /* plane streaming: a block walks its tile plane by plane through a
                                    shared-memory ring, caching some planes in registers / shared
                                    memory */
    PERKS_KERNEL_PER_STEP = 3    /* one launch per step (PERKS_PER_STEP) */
};

/* Creates a stencil over a device-resident domain described by *desc (the
 * library keeps its own copy of the field, two ping-pong buffers and the halo
 * buffers).  Errors: INVALID_ARG (bad extents, radius, offsets outside the
 * radius, npts), UNSUPPORTED (dtype), OUT_OF_MEMORY. */
perks_status perks_stencil_create(perks_context *ctx, const perks_stencil_desc *desc,
                                  perks_stencil **out);
perks_status perks_stencil_destroy(perks_stencil *st);

/* Step trace of the persistent kernel (a tracing aid, not in the paper):
 * with steps > 0 the next persistent runs record, for every block, the
 * %globaltimer value (ns) when it starts and ends its work in each of the
 * first `steps` time steps (and in the prologue, as step -1); steps = 0 turns
 * tracing off.  get_trace copies 2 * (steps + 1) * grid_blocks values of the
 * last traced run, laid out [step + 1][block][start, end], into `host`.
 * Errors: INVALID_ARG (no traced run, capacity too small), OUT_OF_MEMORY. */
perks_status perks_stencil_set_trace(perks_stencil *st, int32_t steps);
perks_status perks_stencil_get_trace(perks_stencil *st, uint64_t *host, int64_t capacity,
                                     int32_t *grid_blocks, int32_t *steps);

/* Autotuner (not in the paper): times candidate plans for `variant` on the
 * stencil's current field -- each as the difference between runs of
 * `probe_steps` (>= 2) and 3 `probe_steps` steps, so that the per-run launch,
 * prologue and epilogue cancel -- the resident-tile kernel with 256 and 512
 * threads and 1 and 2 rows per thread where the domain fits, and the model's
 * own tiling and up to six tilings ranked by tz * (1 + halo fraction), each
 * with registers + shared memory, shared memory only, no cache, or no cache
 * in balanced shares (perks_stencil_plan.balanced), and with 2 or 4 planes
 * per block barrier -- restores the field, installs the fastest plan (as
 * perks_stencil_set_plan would) and returns it with its time per step.
 * Synchronizes `stream`.  Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY,
 * CUDA, BARRIER_TIMEOUT. */
perks_status perks_stencil_autotune(perks_stencil *st, int32_t variant, int32_t probe_steps,
                                    perks_stream stream, perks_stencil_plan *chosen,
                                    double *ms_per_step);

/* Plan override (NULL resets to automatic).  Errors: INVALID_ARG,
 * UNSUPPORTED (the persistent kernel cannot host the requested tiles). */
perks_status perks_stencil_set_plan(perks_stencil *st, const perks_stencil_plan *plan);

/* Copies nx*ny*nz elements of the storage dtype (double / float / bf16 bits
 * as uint16) from `src` into the field; `src_on_device` says whether src is a
 * device (1) or host (0) pointer.  Stream-ordered. */
perks_status perks_stencil_set_field(perks_stencil *st, const void *src, int src_on_device,
                                     perks_stream stream);

/* Advances the field by `steps` Jacobi steps (>= 0) with `variant`:
 *   PERKS_PERSISTENT: one cooperative launch holding the whole time loop
 *     (Listing 1 / Fig. 4), tiles cached in registers + shared memory,
 *     halos through L2;
 *   PERKS_PER_STEP: one launch per step, every step reading and writing the
 *     whole field in HBM (the baseline PERKS is measured against).
 * Both give the same values up to rounding order: with fp32 / bf16 storage
 * every kernel adds a cell's terms in table order by fp32 fused multiply-adds,
 * so all plans and variants give the same bits; with fp64 the order can
 * differ between kernel bodies (the cache-free 3d7pt body with six equal
 * neighbour weights sums the neighbours, then applies the two weights).
 * With opt_out == NULL the
 * call is asynchronous; device errors (BARRIER_TIMEOUT) then surface in
 * perks_stencil_check.  With opt_out != NULL the stream is synchronized and
 * opt_out filled.  Errors: INVALID_ARG, LAUNCH_TOO_LARGE, UNSUPPORTED,
 * BARRIER_TIMEOUT, CUDA. */
perks_status perks_stencil_run(perks_stencil *st, int64_t steps, int32_t variant,
                               perks_stream stream, perks_run_stats *opt_out);

/* Plans a run without launching it (fills *out as perks_stencil_run would). */
perks_status perks_stencil_describe(perks_stencil *st, int64_t steps, int32_t variant,
                                    perks_run_stats *out);

/* Synchronizes `stream` and reports a device-side error of earlier runs on
 * this stencil (BARRIER_TIMEOUT), clearing it. */
perks_status perks_stencil_check(perks_stencil *st, perks_stream stream);

/* Copies the current field out (same element type and layout as set_field). */
perks_status perks_stencil_get_field(perks_stencil *st, void *dst, int dst_on_device,
                                     perks_stream stream);

/* Allocation-free persistent run, for callers that cannot allocate device
 * memory: code running under an external memory-pool manager that owns all
 * device memory, or a latency-critical loop where a cudaMalloc would
 * synchronize the device.  The paper has no counterpart; this entry point
 * exists only for such callers.
 *
 * Computes what perks_stencil_create + set_field + perks_stencil_run(steps,
 * PERKS_PERSISTENT) + get_field would, for the stencil *desc (dtype PERKS_F64
 * or PERKS_F32), without creating a stencil object and without allocating any
 * memory.  `in` and `out` are device pointers on the calling thread's current
 * device, each holding nx*ny*nz elements of the dtype; `in` is only read
 * (in == out updates the field in place; other overlaps are undefined) and
 * `out` receives the field after `steps` steps.
 *
 * Scratch (second ping-pong field, transposed x-edges, barrier counter, error
 * record) is one static device array compiled into the library, about 12 MiB,
 * held on every GPU that loads the library until the process exits.  Limits:
 * nx*ny*nz <= 2^20 cells and the plan's x-edge buffers <= 4 MiB; larger
 * problems (each extent is checked before their product is formed) return
 * PERKS_ERR_INVALID_ARG before any GPU work.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it for
 * the life of the process; make that first call outside any stream capture,
 * and do not use this entry point on a device after cudaDeviceReset (the
 * kept address would be stale).  Every call reuses the same array and clears
 * its counter and error record, so calls whose kernels overlap on the GPU
 * (other streams, other host threads) race.
 *
 * Besides device memory, the call makes no heap allocation on the host
 * either, except that the library's table of compiled kernels is built on
 * the first call in the process that plans any stencil run (once).  No
 * message is formatted or recorded (there is no context).
 *
 * sync == 0: asynchronous, device-side errors are not reported; sync != 0:
 * synchronizes `stream` and returns PERKS_ERR_BARRIER_TIMEOUT if a grid
 * barrier wait ran past 2 s.  Other errors: INVALID_ARG, UNSUPPORTED (shape
 * or dtype without a persistent kernel), LAUNCH_TOO_LARGE, CUDA. */
perks_status perks_stencil_run_noalloc(const perks_stencil_desc *desc, const void *in, void *out,
                                       int64_t steps, perks_stream stream, int32_t sync);

/* ------------------------------------------------------------------------ */
/* Batched stencils: many uneven 2-D domains in one persistent launch         */
/* (Sec. 3 execution model applied to a set of domains; tile assignment and  */
/* cache split from the Sec. 5.2 performance model, refined by timing)       */
/* ------------------------------------------------------------------------ */

typedef struct perks_batch perks_batch;

typedef struct {
    int64_t steps;
    int32_t grid_blocks;
    int32_t tiles;                      /* tiles over all domains */
    int32_t max_tiles_per_block;
    int32_t width_cap;                  /* max tile width in cells (0: kernel limit) */
    int64_t smem_bytes_per_block;
    int64_t cells, cached_cells, halo_cells_per_step;
    double granularity;                 /* target tile cells / (total cells / blocks) */
    double predicted_ms_per_step;       /* model makespan of the chosen plan (ring kernel) */
    double algorithmic_bytes;           /* S (2 N D_uncache + 2 D_cache) + S N H */
    int32_t kernel;                     /* PERKS_BATCH_RING or PERKS_BATCH_STRIP */
    int32_t strip_rows;                 /* strip kernel: output rows per item (0 = automatic) */
} perks_batch_stats;

/* Kernels of the batched persistent launch.
 *   PERKS_BATCH_RING: each block walks its tiles (row ranges of a domain)
 *     through a shared-memory plane ring and caches the rows its shared
 *     memory has room for between steps (the PERKS cache split);
 *   PERKS_BATCH_STRIP: each warp streams its items (a 32-vector-wide column
 *     strip of a domain over a range of rows) through a private ring of rows
 *     with 2R + 1 rows of the stencil in registers; halo cells come from the
 *     previous step's field, so no warp waits for another inside a step; no
 *     cells are cached between steps (fp32 and fp64 storage). */
enum { PERKS_BATCH_RING = 0, PERKS_BATCH_STRIP = 1 };

/* Creates a batch of `ndom` 2-D domains, descs[i] each (all the same dtype;
 * shapes 2d5pt, 2d9pt, 2d25pt or 2ds9pt in any mix; nx a multiple of 16 bytes
 * of cells: 2 for F64, 4 for F32, 8 for BF16).  The library owns two field
 * buffers per domain.  Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY. */
perks_status perks_batch_create(perks_context *ctx, int32_t ndom, const perks_stencil_desc *descs,
                                perks_batch **out);
perks_status perks_batch_destroy(perks_batch *b);
/* Field of domain `dom` in/out (nx*ny elements, layout as perks_stencil_set_field). */
perks_status perks_batch_set_field(perks_batch *b, int32_t dom, const void *src, int src_on_device,
                                   perks_stream stream);
perks_status perks_batch_get_field(perks_batch *b, int32_t dom, void *dst, int dst_on_device,
                                   perks_stream stream);
/* Advances every domain by `steps` steps: PERKS_PERSISTENT = one cooperative
 * launch for all domains; PERKS_PER_STEP = one launch per domain per step
 * (baseline).  opt_out as in perks_stencil_run. */
perks_status perks_batch_run(perks_batch *b, int64_t steps, int32_t variant, perks_stream stream,
                             perks_batch_stats *opt_out);
/* Autotuner: ranks the ring kernel's tile granularities and width caps with
 * the performance model, times the best few and the strip kernel with items
 * of 32 to 256 rows for `probe_steps` steps each (0: model only;
 * the fields are restored afterwards) and keeps the fastest plan.  Allocates
 * a temporary copy of the fields while probing.  *chosen may be NULL. */
perks_status perks_batch_autotune(perks_batch *b, int64_t probe_steps, perks_stream stream,
                                  perks_batch_stats *chosen);
/* Fixes the plan parameters instead (granularity > 0, width_cap >= 0) and
 * selects the ring kernel they apply to. */
perks_status perks_batch_set_plan(perks_batch *b, double granularity, int32_t width_cap);
/* Selects the kernel (PERKS_BATCH_RING / PERKS_BATCH_STRIP; the strip kernel
 * is the default where it is compiled) and, for the strip kernel, the output
 * rows per item (0 = automatic).  The autotuner times both kernels.  Errors:
 * INVALID_ARG, UNSUPPORTED (no strip kernel for the dtype). */
perks_status perks_batch_set_kernel(perks_batch *b, int32_t kernel, int32_t strip_rows);

/* ------------------------------------------------------------------------ */
/* Conjugate gradient: Sec. 2.2.2 (algorithm), Sec. 4.3 (PERKS port)          */
/* ------------------------------------------------------------------------ */

enum {
    PERKS_CG_FP64 = 0,        /* fp64 CG, one persistent launch */
    PERKS_CG_FP32_IR = 1,     /* fp32 inner CG + fp64 true residual and refinement, one launch */
    PERKS_CG_FP64_MULTI = 2   /* fp64 CG, several launches per iteration (baseline) */
};

/* Builds a CSR operator with n rows, nnz nonzeros, int32 row pointers
 * (n+1), int32 column indices (nnz, sorted or not within a row) and fp64
 * values (nnz).  A must be symmetric positive definite for CG; this is not
 * checked.  `on_device` says where the three arrays live.  The library keeps
 * device copies (and an fp32 copy of the values for PERKS_CG_FP32_IR).
 * Errors: INVALID_ARG (n < 1, nnz < 0, NULL), OUT_OF_MEMORY, CUDA. */
perks_status perks_csr_create(perks_context *ctx, int32_t n, int64_t nnz, const int32_t *rowptr,
                              const int32_t *col, const double *val, int on_device,
                              perks_op **out);
perks_status perks_op_destroy(perks_op *op);

/* SpMV variant used inside CG and by perks_csr_spmv.  All split the rows
 * over blocks by the merge-path diagonal search (computed once).  Inside a
 * block, ROWVEC gives each row to 4 lanes with direct coalesced loads and one
 * fused multiply-add per nonzero (default); MERGE is the two-level merge-based
 * SpMV of Sec. 4.3 (thread-level diagonal search over staged tiles, which
 * also keeps A in shared memory when a block's slice fits); SEG stages the
 * multiplied vector in shared memory one column segment at a time, together
 * with the block's nonzeros of that segment (bulk asynchronous copies, two
 * buffers), so every gather is a shared-memory access -- not in the paper;
 * its layout is built on the GPU when the kind is first selected (about 16
 * bytes per nonzero).  Errors: INVALID_ARG; UNSUPPORTED for SEG when a block
 * would own more than 8192 rows or a block's nonzeros in one 4096-column
 * segment exceed 2048. */
enum { PERKS_SPMV_ROWVEC = 0, PERKS_SPMV_MERGE = 1, PERKS_SPMV_SEG = 2 };
perks_status perks_op_set_spmv(perks_op *op, int32_t kind);

/* Vector cache of the persistent CG with the ROWVEC SpMV (the caching of the
 * residual vector of Sec. 4.3.2): each block keeps its rows of vectors only
 * it touches in shared memory for the whole solve -- level 1: r (the inner
 * r for FP32_IR); level 2: x, r and q (inner r, d and q); p, which every
 * block gathers, stays in global memory.  Level 0 (default) keeps every
 * vector in global memory.  A level takes effect when the largest block's
 * rows fit at 24 bytes per row with all blocks co-resident.  Results are
 * identical at every level.  On GB300 the cache is slower (n = 2^20 to 1e-8:
 * 9.7 ms without, 12.6 ms at level 2): the shared memory it takes comes out
 * of the unified L1, which holds the SpMV's gathers in flight.  Errors:
 * INVALID_ARG. */
perks_status perks_op_set_vector_cache(perks_op *op, int32_t level);
/* The level the next persistent solve of `op` runs with (0: none). */
int32_t perks_op_vector_cache_active(const perks_op *op);

/* y = A x for device vectors of n doubles (one launch). */
perks_status perks_csr_spmv(perks_op *op, const double *x, double *y, perks_stream stream);

typedef struct {
    int32_t iterations;          /* CG recurrence iterations (fp32 inner ones for FP32_IR) */
    int32_t outer_iterations;    /* restarts (FP64) or refinement steps (FP32_IR) */
    double true_rel_residual;    /* ||b - A x|| / ||b|| in fp64, recomputed on the GPU */
    int32_t status;              /* same value the call returns */
    int32_t grid_blocks, threads_per_block;
    double bytes_per_iteration;  /* algorithmic bytes of one recurrence iteration */
    double *trace;               /* optional host array of 3*trace_len doubles:
                                    (alpha_k, beta_k, <r_{k+1}, r_{k+1}>) per iteration */
    int32_t trace_len;
} perks_cg_stats;

/* Solves A x = b to ||r|| <= rtol ||b||.  `b` (n doubles) is read, `x` (n
 * doubles) holds x0 on entry and the solution on exit; both are device
 * pointers when on_device = 1, host pointers otherwise.  `max_iter` bounds
 * the recurrence iterations; for FP32_IR `inner_rtol` is the inner solves'
 * relative tolerance, 0 = automatic: sqrt(rtol) clamped to [1e-6, 0.1], so
 * that two refinement steps reach rtol (ignored for the other modes).  On exit the true residual is
 * recomputed in fp64; above tolerance the solver restarts (FP64) or refines
 * again (FP32_IR) while iterations remain.  With stats == NULL the call is
 * asynchronous and returns 0 once launched; the outcome is then read by
 * perks_cg_last_result.  Errors: INVALID_ARG, LAUNCH_TOO_LARGE,
 * NOT_CONVERGED, BREAKDOWN, BARRIER_TIMEOUT, CUDA. */
perks_status perks_cg_solve(perks_op *op, const double *b, double *x, double rtol,
                            int32_t max_iter, int32_t mode, double inner_rtol, int on_device,
                            perks_stream stream, perks_cg_stats *stats);

/* Synchronizes `stream` and fills *stats (may be NULL) with the outcome of
 * the last solve; returns that solve's status. */
perks_status perks_cg_last_result(perks_op *op, perks_stream stream, perks_cg_stats *stats);

/* ------------------------------------------------------------------------ */
/* Batched variable-coefficient Poisson (learned warm start workload)         */
/* ------------------------------------------------------------------------ */
/* -div(k grad u) = f on nprob grids of nx*ny cells (5-point finite volumes,
 * h = 1; face coefficient = harmonic mean of the two cells' k; Dirichlet 0
 * through a ghost cell with the boundary cell's k), each solved by the CG of
 * Sec. 2.2.2 in ONE persistent launch: each block owns a problem at a time
 * and runs its whole CG loop with block-level reductions (the problems are
 * independent, so no grid barrier is needed).  Not in the paper: this is the
 * workload of the learned warm start. */
typedef struct perks_poisson perks_poisson;

typedef struct {
    int32_t problems;
    int32_t grid_blocks;
    int32_t max_iterations;
    double mean_iterations;
    double max_true_rel_residual;     /* worst ||b - A x|| / ||b|| (fp64) */
    int32_t *iterations;              /* optional host array, `capacity` entries */
    double *true_rel_residual;        /* optional host array, `capacity` entries */
    int32_t capacity;
} perks_poisson_stats;

/* k: nprob*ny*nx coefficients (x fastest, problem slowest), > 0; on_device
 * says where k lives.  The library keeps the face coefficients and work
 * vectors.  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
perks_status perks_poisson_create(perks_context *ctx, int32_t nx, int32_t ny, int32_t nprob,
                                  const double *k, int on_device, perks_poisson **out);
perks_status perks_poisson_destroy(perks_poisson *p);
/* y = A v for every problem; v, y: device arrays of nprob*nx*ny doubles. */
perks_status perks_poisson_apply(perks_poisson *p, const double *v, double *y, perks_stream stream);
/* Scales each problem's guess x (device, nprob*nx*ny doubles, in place) by
 * alpha = <x, b> / <x, A x>, the multiple of x closest to the solution of
 * A u = b in the A-norm (a one-dimensional Galerkin projection): for a
 * learned warm start, an error in its overall amplitude costs no CG
 * iterations.  A problem whose <x, A x> is not positive and finite (x = 0)
 * keeps its x.  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
perks_status perks_poisson_scale_guess(perks_poisson *p, const double *b, double *x, perks_stream stream);
/* Solves every problem to ||r|| <= rtol ||b|| from x (device arrays of
 * nprob*nx*ny doubles; x holds x0 and receives the solutions).  With stats
 * the stream is synchronized and the per-problem outcome reported; the call
 * then returns the first failing problem's status. */
perks_status perks_poisson_solve(perks_poisson *p, const double *b, double *x, double rtol,
                                 int32_t max_iter, perks_stream stream, perks_poisson_stats *stats);
/* Block shape of the 4-rows-per-pass kernel (perks_poisson_set_rows_per_pass):
 * 512 threads (one block per SM, default) or 256 (two per SM: twice as many
 * blocks, half the loads in flight per block).  With one block per problem
 * a batch finishes with its slowest problem running alone, where the larger
 * block is faster (256 problems of 512^2 to 1e-8, before the diagonal was
 * precomputed: 23.6 s vs 31.8 s).  Errors: INVALID_ARG. */
perks_status perks_poisson_set_block_threads(perks_poisson *p, int32_t threads);
/* Blocks per problem: 1, 2, 4 or 8, or 0 (the default: for problems of
 * 65536 cells and more 8 with one row per pass, 4 with four, and 1 below;
 * 256 problems of 512^2 to 1e-8 at four rows per pass take 20.2 s with C =
 * 1, 16.4 s with 2 and 15.9 s with 4).  With C > 1 each problem's
 * rows are split over a group of C blocks that meet at a bounded barrier of
 * their own after every p update and in every dot product (the group's block
 * sums are added in rank order, so all its blocks take the same decisions);
 * the launch is cooperative.  A batch ends with its hardest problem running
 * alone; a group runs it up to C times faster, at the price of fewer problems
 * in flight.  Iteration counts may differ from C = 1 by rounding (another
 * summation order).  A barrier wait past the context's timeout ends the solve
 * with BARRIER_TIMEOUT (reported when stats are requested).  Errors:
 * INVALID_ARG. */
perks_status perks_poisson_set_group(perks_poisson *p, int32_t blocks);
/* Rows of a grid column each thread takes per pass of the matvec: 1
 * (default: 64 registers, two 512-thread blocks per SM, twice the warps to
 * hide load latency) or 4 (each column value and face loaded once for 4
 * cells, 128 registers, one block per SM, or two of 256 threads, as
 * perks_poisson_set_block_threads says).  256 problems of 512^2 to 1e-8,
 * automatic groups: 13.4 s with 1, 15.9 s with 4.  The block shape of
 * perks_poisson_set_block_threads applies with 4 only.  Errors:
 * INVALID_ARG. */
perks_status perks_poisson_set_rows_per_pass(perks_poisson *p, int32_t rows);


/* ------------------------------------------------------------------------ */
/* Learned warm start for the Poisson workload                                */
/* ------------------------------------------------------------------------ */
/* A 4-layer convolutional network, u0 = scale * N(log k, f): 3x3 convolutions
 * (2 -> 32 -> 32 -> 32 -> 1 channels, dilations d[0..3], zero padding), ReLU
 * after the first three; activations stored in BF16 (or F32), products
 * accumulated in fp32, fp32 master weights trained by Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) on the mean squared error against u / scale.
 * Parameter layout, per layer l: W_l[cout][cin][3][3] then b_l[cout].  Not
 * in the paper: the warm start only chooses x0, CG still solves to the
 * requested tolerance. */
typedef struct perks_warmnet perks_warmnet;

/* dilations: 4 values in 1..16 (NULL = {1, 2, 4, 8}); storage PERKS_BF16 or
 * PERKS_F32; weights He-initialised from `seed`, biases 0.  Errors:
 * INVALID_ARG, OUT_OF_MEMORY, CUDA. */
perks_status perks_warmnet_create(perks_context *ctx, const int32_t *dilations, int32_t storage,
                                  uint64_t seed, perks_warmnet **out);
perks_status perks_warmnet_destroy(perks_warmnet *net);
int32_t perks_warmnet_num_params(const perks_warmnet *net);
/* Copy the fp32 parameters to / from a host array of num_params floats. */
perks_status perks_warmnet_get_params(perks_warmnet *net, float *host);
perks_status perks_warmnet_set_params(perks_warmnet *net, const float *host);
/* Coarse-grid mode (factor 1..32, default 1): the inputs log k and f are
 * averaged over factor x factor blocks, the network runs on that coarser
 * grid (training targets u averaged the same way), and predict() returns the
 * bilinear interpolation of its output at the fine cell centres; grids must
 * then be divisible by the factor (else INVALID_ARG). */
perks_status perks_warmnet_set_pool(perks_warmnet *net, int32_t factor);
/* BF16 storage only: run the two 32 -> 32 layers of the forward pass as
 * implicit GEMMs on the tensor cores (tcgen05.mma, fp32 accumulation in
 * tensor memory; default) or on the CUDA cores (enable = 0). */
perks_status perks_warmnet_set_tensor_cores(perks_warmnet *net, int32_t enable);
/* Output scale (> 0): the network predicts u / scale. */
perks_status perks_warmnet_set_scale(perks_warmnet *net, float scale);
float perks_warmnet_get_scale(const perks_warmnet *net);
/* u = scale * N(log k, f) for nimg images of ny*nx cells; k, f, u are device
 * arrays of nimg*ny*nx doubles (x fastest).  Asynchronous on `stream`. */
perks_status perks_warmnet_predict(perks_warmnet *net, int32_t nimg, int32_t ny, int32_t nx,
                                   const double *k, const double *f, double *u, perks_stream stream);
/* Loss L = mean((N(log k, f) - u / scale)^2) and dL/dparams (host arrays;
 * either may be NULL); synchronizes `stream`. */
perks_status perks_warmnet_gradient(perks_warmnet *net, int32_t nimg, int32_t ny, int32_t nx,
                                    const double *k, const double *f, const double *u,
                                    float *grad_host, float *loss_host, perks_stream stream);
/* One Adam step with learning rate lr on the batch (k, f, u); the loss before
 * the step goes to *loss_host when non-NULL (then the stream is synchronized). */
perks_status perks_warmnet_train_step(perks_warmnet *net, int32_t nimg, int32_t ny, int32_t nx,
                                      const double *k, const double *f, const double *u, float lr,
                                      perks_stream stream, float *loss_host);
/* Trains for `epochs` passes over nimg pairs (k, f) -> u (device arrays as
 * in predict), in minibatches of `batch` consecutive images visited in an
 * order shuffled per epoch from `seed`, one Adam step (rate lr) per
 * minibatch.  auto_scale = 1 first sets scale = rms(u).  epoch_loss (host,
 * `epochs` floats, may be NULL) receives each epoch's mean minibatch loss.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
perks_status perks_warmnet_fit(perks_warmnet *net, int32_t nimg, int32_t ny, int32_t nx,
                               const double *k, const double *f, const double *u, int32_t batch,
                               int32_t epochs, float lr, int32_t auto_scale, uint64_t seed,
                               perks_stream stream, float *epoch_loss);

#ifdef __cplusplus
}
#endif

#endif /* PERKS_H */
