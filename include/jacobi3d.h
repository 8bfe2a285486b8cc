/*
 * jacobi3d.h -- C ABI of the GB300 Jacobi3D library (libjacobi3d.so).
 *
 * The library runs the paper's Jacobi3D proxy application ("Improving
 * Scalability with GPU-Aware Asynchronous Tasks", Choi, Richards, Kale):
 * a 3D grid overdecomposed into blocks that each carry a one-cell ghost
 * layer and two copies of their data (Section III-C), updated every
 * iteration after the halos of the previous iteration have been packed,
 * exchanged with the six face neighbours and unpacked (Section II-A,
 * Figs. 1 and 3). All blocks live in one GPU's HBM; the exchange is a
 * device-to-device copy or a direct read of the neighbour's face.
 *
 * Conventions
 *   - Global interior arrays are x fastest: cell (i, j, k) of an
 *     nx x ny x nz grid is element i + nx*(j + ny*k).
 *   - Faces and boundary values are ordered -x, +x, -y, +y, -z, +z.
 *   - The update of an interior cell is the mean of itself and its six face
 *     neighbours; outside the global grid the neighbours are the Dirichlet
 *     values bc[6], constant across iterations.
 *   - Every call returns JAC_OK (0) or a negative JAC_E* code; no call
 *     aborts, throws or exits. jac_strerror() names a code; jac_last_error()
 *     gives a human-readable message for the calling thread's last failure.
 *   - Host pointers are borrowed for the duration of the call only. Device
 *     memory of a context is owned by the library and freed by
 *     jac_destroy().
 *   - Calls on one context must not run concurrently from several host
 *     threads. Work is ordered on the context's CUDA stream.
 */
#ifndef JACOBI3D_H
#define JACOBI3D_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Codes and enums                                                     */
/* ------------------------------------------------------------------ */

#define JAC_OK 0
#define JAC_EINVAL (-1)   /* bad argument: null pointer, size, dims, mode   */
#define JAC_ENOMEM (-2)   /* a device or host allocation failed             */
#define JAC_ECUDA (-3)    /* a CUDA runtime call failed                     */
#define JAC_ETIMEOUT (-4) /* a device-side wait gave up (bounded spin)      */
#define JAC_EBUDGET (-5)  /* the request exceeds the configured HBM budget  */
#define JAC_ESTATE (-6)   /* call not valid in the context's current state  */

typedef enum { JAC_F64 = 0, JAC_F32 = 1 } jac_dtype;

/* How one iteration is issued (paper Sections III-A and III-D):
 *  UNFUSED    per block: 6 pack kernels, 6 device-to-device halo copies into
 *             the neighbours' receive buffers, 6 unpack kernels into the
 *             ghost layer and 1 update kernel, on per-block streams (packing,
 *             copies and unpacking on high-priority streams, the update on a
 *             low-priority one, Section III-A), ordered with events.
 *  FUSED      one kernel per iteration for all blocks: unpack, update and
 *             pack fused (strategy C of Section III-D1) by reading each ghost
 *             face straight from the neighbour block.
 *  GRAPH      the UNFUSED iteration captured once as a CUDA graph per
 *             pointer parity, the two graphs launched alternately
 *             (Section III-D2).
 *  PERSISTENT one launch runs all requested iterations for all blocks; each
 *             block waits only for its six neighbours to finish the previous
 *             iteration (per-block iteration counters, the device form of
 *             the reference numbers of Section II-A), with bounded waits.
 *  GRAPH_FUSED the FUSED kernel captured as two alternating graphs.
 *  SPLIT      the UNFUSED flow with the manual overlap of Section II-A
 *             (Fig. 1): per block the interior update (cells 1 .. b-2 on
 *             every axis, which read no halo) runs on the low-priority
 *             compute stream while the high-priority communication stream
 *             packs, exchanges and unpacks the halos (the priorities of
 *             Section III-A); the exterior layer is updated after the
 *             unpack. A comparison form: per-cell updates, not the tile
 *             engines.                                                    */
typedef enum {
    JAC_MODE_UNFUSED = 0,
    JAC_MODE_FUSED = 1,
    JAC_MODE_GRAPH = 2,
    JAC_MODE_PERSISTENT = 3,
    JAC_MODE_GRAPH_FUSED = 4,
    JAC_MODE_SPLIT = 5
} jac_mode;

/* Rounding of the binary64 mean (binary32 contexts always use SEQ):
 *  SEQ    left-to-right sum c, -x, +x, -y, +y, -z, +z, each addition
 *         rounded to nearest even, then a correctly rounded division by 7,
 *         in the GPU's binary64 units.
 *  EXACT  the exact sum of the seven values divided by 7 and rounded once to
 *         nearest even (the correctly rounded mean), computed in integer
 *         arithmetic.                                                     */
typedef enum { JAC_ARITH_SEQ = 0, JAC_ARITH_EXACT = 1 } jac_arith;

typedef struct jac_ctx jac_ctx;

typedef struct {
    int64_t dims[3];         /* nx, ny, nz                                   */
    int32_t block[3];        /* requested block dims bx, by, bz              */
    int32_t nblocks[3];      /* blocks per axis                              */
    int32_t dtype;           /* jac_dtype                                    */
    int32_t mode;            /* jac_mode                                     */
    int32_t arith;           /* jac_arith                                    */
    int32_t persistent_ctas; /* CTAs of the persistent launch (0 until used) */
    int64_t iterations;      /* iterations completed (enqueued) so far       */
    int64_t device_bytes;    /* device memory held by the context            */
    int64_t kernel_launches; /* kernels this context has launched so far     */
    int32_t n_instances;     /* grids held by the context                    */
    int32_t tile_w;          /* tile width of the update engine (16/32/64)  */
    int32_t zdepth;          /* planes per work unit (0: whole block)        */
    int32_t n_units;         /* work units (tile x z-chunk) per iteration    */
    int32_t n_blocks;        /* blocks over all instances                    */
} jac_info_t;

/* Result of jac_autotune: the chosen configuration and every trial. */
typedef struct {
    int32_t tile_w;                 /* chosen tile width                    */
    int32_t zdepth;                 /* chosen z depth (0: whole block)      */
    double ms_per_iter;             /* its time per iteration               */
    int32_t n_trials;
    int32_t trial_tile_w[16];
    int32_t trial_zdepth[16];
    double trial_ms_per_iter[16];
    int32_t n_classes;           /* block-width classes refined (0: one width for all blocks) */
    int32_t class_block_x[16];   /* a class: blocks of this x extent ...                      */
    int32_t class_tile_w[16];    /* ... run with this tile width                              */
    double ms_per_iter_classes;  /* ms per iteration after the per-class refinement           */
} jac_tune_t;

/* ------------------------------------------------------------------ */
/* Memory hook                                                         */
/* ------------------------------------------------------------------ */

/* Route the library's device allocations through a caller's allocator (the
 * Python binding installs PyTorch's caching allocator). alloc returns a
 * device pointer of at least `bytes` bytes, 256-byte aligned, usable on
 * `stream`, or NULL; free releases it. Passing NULLs restores the default
 * (cudaMallocAsync / cudaFreeAsync on the context's stream). Applies to
 * contexts created afterwards. Not thread-safe against concurrent creates. */
typedef void *(*jac_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*jac_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
int jac_set_allocator(jac_alloc_fn alloc, jac_free_fn free_fn, void *user);

/* ------------------------------------------------------------------ */
/* Host buffers                                                        */
/* ------------------------------------------------------------------ */

/* Page-locked, zero-filled host memory of at least `bytes` bytes for the
 * host forms of jac_write / jac_read (and any other host<->device copy),
 * laid out for the host link. A request of 64 MiB or more is backed by the
 * kernel's transparent huge pages where it offers them on request: anonymous
 * memory aligned to the huge-page size, advised MADV_HUGEPAGE, placed
 * preferably on the current GPU's nearest host NUMA node, touched, then
 * registered with cudaHostRegister, when the kernel gives (nearly) all of it
 * huge pages (else the memory comes from cudaHostAlloc: registered base pages
 * copy more slowly than the driver's pinned memory). A copy then needs one
 * address translation per huge page instead of one per base page. On GB300 (64 KiB
 * base pages, 512 MiB huge pages) a pinned 1 GiB buffer of base pages that
 * has not been copied for a second or more takes 80-210 ms for its next
 * copy, about 7 us per page translation, and 5.1 ms for the copies after it;
 * a huge-page buffer takes 5.1 ms every time. Smaller requests, and systems
 * without transparent huge pages, get cudaHostAlloc memory. Both are
 * registered as portable (pinned for every CUDA context of the process).
 * Needs a CUDA device. Returns NULL on failure (jac_last_error says why).
 * Thread-safe. */
void *jac_host_alloc(size_t bytes);

/* Release memory from jac_host_alloc. NULL is ignored; any other pointer
 * jac_host_alloc did not return gives JAC_EINVAL. */
int jac_host_free(void *p);

/* What backs a pointer jac_host_alloc returned: 1 huge pages (registered),
 * 0 cudaHostAlloc memory, -1 a pointer it did not return. */
int jac_host_alloc_kind(const void *p);

/* ------------------------------------------------------------------ */
/* Context lifecycle                                                   */
/* ------------------------------------------------------------------ */

/* Create a context for one global grid.
 * The paper's statement of the problem: a global 3D grid decomposed into
 * cuboid blocks (Section IV-A, overdecomposition factor), each block with
 * one-cell ghost layers and two copies of its data (Section III-C).
 *   out      receives the new context (set to NULL on failure).
 *   nx,ny,nz global interior dims, each >= 1.
 *   bx,by,bz requested block dims, 1 <= b* <= n*, b* <= 256. An axis of n
 *            cells is split into ceil(n / b) blocks whose sizes differ by at
 *            most one, the larger ones first.
 *   dtype    JAC_F64 or JAC_F32: storage and arithmetic type.
 *   bc       6 finite Dirichlet values (-x, +x, -y, +y, -z, +z); for F32
 *            they are rounded to nearest binary32. |bc| <= 1e300.
 *   stream   a cudaStream_t (may be NULL for the legacy default stream) on
 *            which all of the context's work is ordered.
 * The interior starts at 0. Fails with JAC_EINVAL on bad arguments,
 * JAC_ENOMEM if device memory runs out, JAC_ECUDA on other CUDA errors. */
int jac_create(jac_ctx **out, int64_t nx, int64_t ny, int64_t nz, int32_t bx, int32_t by,
               int32_t bz, int32_t dtype, const double bc[6], void *stream);

/* Create a context holding n_inst independent grids that are stored in one
 * pool, described by one block table and advanced by the same launches
 * (batching several problems into one persistent or fused launch; the
 * paper's overdecomposition, Section IV-A, applied across problems).
 *   dims     3*n_inst values: nx, ny, nz of grid i at dims[3i .. 3i+2].
 *   bc       6*n_inst Dirichlet values, grid i at bc[6i .. 6i+5].
 *   others   as jac_create; every grid uses the same requested block dims
 *            (each axis of each grid is split as jac_create describes).
 * Dense host/device arrays of the whole context hold the grids back to back
 * in instance order, each x fastest. */
int jac_create_batch(jac_ctx **out, int32_t n_inst, const int64_t *dims, int32_t bx, int32_t by,
                     int32_t bz, int32_t dtype, const double *bc, void *stream);

/* Release the context and all of its device memory after its stream has
 * drained. NULL is accepted. */
int jac_destroy(jac_ctx *h);

/* Select how iterations are issued (jac_mode). Default JAC_MODE_PERSISTENT.
 * Any mode may follow any other; the grid state carries over. */
int jac_set_mode(jac_ctx *h, int32_t mode);

/* Select the binary64 rounding (jac_arith); default JAC_ARITH_EXACT.
 * JAC_EINVAL for F32 contexts unless arith == JAC_ARITH_SEQ. */
int jac_set_arith(jac_ctx *h, int32_t arith);

/* ------------------------------------------------------------------ */
/* Data in and out                                                     */
/* ------------------------------------------------------------------ */

/* Set the interior from a host array of n_cells = nx*ny*nz binary64 values
 * (x fastest). Values must be finite with magnitude <= 1e300 (<= 3e38 for
 * F32 contexts, which round them to nearest). They are copied to a device
 * staging buffer and checked there before anything is overwritten: a bad
 * value gives JAC_EINVAL naming the lowest bad index (jac_last_error) and
 * leaves the grid as it was. Synchronises; the host buffer may be reused on
 * return. Resets the iteration count. */
int jac_write(jac_ctx *h, const double *host, size_t n_cells);

/* As jac_write, from a host binary32 array (F32 contexts only: exact; values
 * must be finite). */
int jac_write_f32(jac_ctx *h, const float *host, size_t n_cells);

/* As jac_write, from device memory already on this GPU: `dev` holds n_cells
 * values of type `dtype` (which must equal the context's dtype), x fastest.
 * The values are checked as for jac_write (binary32: finite) before the grid
 * is touched, which synchronises the context's stream. */
int jac_write_device(jac_ctx *h, const void *dev, size_t n_cells, int32_t dtype);

/* Copy the interior to a host array of n_cells binary64 values (x fastest;
 * F32 values are widened exactly). Synchronises the context's stream and
 * returns JAC_ETIMEOUT if a device wait gave up since the last sync. */
int jac_read(jac_ctx *h, double *host, size_t n_cells);

/* As jac_read into a binary32 host array (F32 contexts only). */
int jac_read_f32(jac_ctx *h, float *host, size_t n_cells);

/* Gather the interior into device memory `dev` (n_cells values of the
 * context's dtype, x fastest). Stream-ordered, no host sync. */
int jac_read_device(jac_ctx *h, void *dev, size_t n_cells, int32_t dtype);

/* ------------------------------------------------------------------ */
/* Iteration and residual                                              */
/* ------------------------------------------------------------------ */

/* Enqueue n_iters >= 0 Jacobi iterations (paper Section II-A: halo
 * exchange then update, two buffers swapped each iteration, Section III-C)
 * in the selected mode. Asynchronous and stream-ordered: no host sync. */
int jac_iterate(jac_ctx *h, int64_t n_iters);

/* rho(u) = sqrt( sum over interior cells of L^2 ),
 * L = xm + xp + ym + yp + zm + zp - 6c evaluated exactly. Per work unit,
 * L^2 is summed exactly and rounded once to binary64 when every value the
 * unit reads lies within the exact range of the integer form: binary64
 * grids, positive values within nine binades of the grid's largest
 * exponent, the grid's largest value between 2^-440 and 2^460 or so;
 * binary32 grids, values within 21 binades of the grid's largest, that
 * largest between 2^-100 and 2^125. Other units (and blocks of odd x extent)
 * round L once to binary64 and sum the squares per thread (binary64: fused
 * multiply-adds; binary32: exactly, then rounded), combining the thread
 * sums by a fixed tree. The units' partials are summed in unit order. That
 * order is fixed by the grid, the block dims, the tile width and z depth, and
 * the unit split the runtime derives from the device's SM count and
 * occupancy: repeated calls on one device and configuration give the same
 * bits, other configurations agree within 1e-12 relative. The paper runs a
 * fixed iteration count and prints no residual (Section IV-A); this is the
 * convergence measure the library adds. Synchronises the stream;
 * JAC_ETIMEOUT as for jac_read. */
int jac_residual(jac_ctx *h, double *out);

/* Enqueue the residual computation and write rho into device memory
 * `dev_out` (one double). Stream-ordered, no host sync. For a batch context
 * rho covers all grids: sqrt of the sum over every grid's cells. */
int jac_residual_device(jac_ctx *h, double *dev_out);

/* Enqueue n_iters >= 0 iterations as jac_iterate does, together with the
 * residual of the grid before every `every`-th of them (every >= 1):
 * dev_out[j] = rho(u^(k0 + j * every)) for j = 0 .. ceil(n_iters / every) - 1,
 * k0 the iteration count at the call; dev_out is device memory of that many
 * doubles (unused when n_iters = 0). In the fused and graph-fused modes
 * (binary32, or binary64 with JAC_ARITH_EXACT) each residual comes from the
 * update launch that reads that grid (kernel fusion, Section III-D1: one
 * launch, no second pass over the grid); other modes and the sequential rule
 * enqueue jac_residual_device before the iteration. Either way dev_out[j] has
 * the bits jac_residual gives for that grid. Stream-ordered, no host sync;
 * JAC_EINVAL for n_iters < 0,
 * every < 1 or a null dev_out, JAC_ESTATE without a resident grid. */
int jac_iterate_residual(jac_ctx *h, int64_t n_iters, int64_t every, double *dev_out);

/* Per-grid residuals of a batch context: out[i] = rho of grid i, same
 * definition as jac_residual. The host form synchronises; the device form
 * writes n_instances doubles to dev_out, stream-ordered. */
int jac_residual_instances(jac_ctx *h, double *out);
int jac_residual_instances_device(jac_ctx *h, double *dev_out);

/* Write or read one grid of a batch context (n_cells = that grid's cells,
 * x fastest); as jac_write / jac_write_device / jac_read /
 * jac_read_device otherwise. Writing resets that grid's frame only and does
 * not change the iteration count. */
int jac_write_instance(jac_ctx *h, int32_t i, const double *host, size_t n_cells);
int jac_write_instance_device(jac_ctx *h, int32_t i, const void *dev, size_t n_cells, int32_t dtype);
int jac_read_instance(jac_ctx *h, int32_t i, double *host, size_t n_cells);
int jac_read_instance_device(jac_ctx *h, int32_t i, void *dev, size_t n_cells, int32_t dtype);

/* Tile shape of the update engine: 512 threads over tile_w x (512/tile_w)
 * columns (binary64) or tile_w x (1024/tile_w) columns (binary32, two per
 * thread), tile_w 16, 32 or 64, each work unit covering zdepth planes of a
 * block (0: all of them). Clears the per-class widths. Results do not depend
 * on it. Synchronises. */
int jac_set_tile(jac_ctx *h, int32_t tile_w, int32_t zdepth);

/* Tile width for the blocks whose x extent is block_x (a block-width class),
 * overriding jac_set_tile's width for them; tile_w 0 removes the override.
 * Results do not depend on it. Synchronises. */
int jac_set_tile_class(jac_ctx *h, int32_t block_x, int32_t tile_w);

/* Autotuner: time trial_iters iterations of the current mode for every tile
 * width and z depth and keep the fastest; when the blocks come in several x
 * extents, then try the other widths class by class (largest classes first,
 * at most 16) and keep each change that makes the whole launch faster.
 * Reports the choice in *result (may be NULL) and restores the grid and
 * iteration count exactly as they were. Needs temporary device memory for
 * one copy of the block storage. Synchronises. */
int jac_autotune(jac_ctx *h, int32_t trial_iters, jac_tune_t *result);

/* Wait for the context's stream and report a device-side wait timeout
 * (JAC_ETIMEOUT) or a CUDA error (JAC_ECUDA). */
int jac_sync(jac_ctx *h);

/* Describe the context. */
int jac_info(jac_ctx *h, jac_info_t *info);

/* Residual rho of a dense grid held by the caller, computed without
 * allocating memory. The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc (or any allocator) where they need
 * the residual, e.g. inside a step of a framework that forbids allocation,
 * while a memory pool is locked, or from a callback that must not block on
 * the allocator.
 *   u        device pointer: nx*ny*nz values of `dtype` (JAC_F64 or
 *            JAC_F32), x fastest, owned by the caller.
 *   bc       6 finite Dirichlet values (-x, +x, -y, +y, -z, +z); binary32
 *            grids use them rounded to binary32.
 *   out      device pointer to one double, receives rho (same definition
 *            as jac_residual).
 *   stream   cudaStream_t (NULL: legacy default stream); stream-ordered,
 *            no host sync. The kernels run on the stream's device; the
 *            calling thread's current device is the same after the call as
 *            before it.
 * Arithmetic: L exact, rounded once to binary64, accumulated in binary64 by
 * fused multiply-adds (acc = fma(L, L, acc)) per column over z, then a fixed
 * tree; binary32 values are widened exactly. The order differs from
 * jac_residual's, so the two agree within 1e-12 relative, not bit for bit.
 * Scratch: the per-CTA partial sums live in a fixed 65536-double (512 KiB)
 * static device array of the library, held by every GPU that loads the
 * library until the process exits. A grid needing more than 65536 partials
 * (ceil(nx/32) * ceil(ny/8) > 65536) is rejected with JAC_EINVAL. The call
 * makes no cudaMalloc/cudaFree or other allocation. Its first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. All calls share the array,
 * which keeps the last call's contents: calls whose kernels overlap on the
 * GPU race and must be serialised by the caller.
 * Returns JAC_EINVAL on bad arguments or sizes, JAC_ECUDA on CUDA errors. */
int jac_residual_dense_noalloc(const void *u, int32_t dtype, int64_t nx, int64_t ny, int64_t nz,
                               const double bc[6], double *out, void *stream);

/* ------------------------------------------------------------------ */
/* Pools: grids that join and leave                                    */
/* ------------------------------------------------------------------ */

/* Bytes of block storage a grid of `dims` needs with these block dims and
 * dtype (both buffers, ghost layers and row padding). */
int jac_storage_bytes(const int64_t dims[3], int32_t bx, int32_t by, int32_t bz, int32_t dtype, int64_t *bytes);

/* An empty context with `capacity_bytes` of block storage and up to
 * `max_grids` grid slots. Grids are added and removed between launches
 * (jac_pool_add / jac_pool_remove); a resident grid's storage never moves,
 * and every launch (fused or persistent forms only) advances all resident
 * grids. Slots index the per-grid calls (jac_write_instance, ...,
 * jac_residual_instances, whose output has one entry per slot, NaN for a
 * free slot). */
int jac_create_pool(jac_ctx **out, int32_t dtype, int64_t capacity_bytes, int32_t max_grids, int32_t bx,
                    int32_t by, int32_t bz, void *stream);

/* Make a grid resident: JAC_EBUDGET if no slot or no free region of the
 * pool fits it. Its interior starts at 0 until written. */
int jac_pool_add(jac_ctx *h, const int64_t dims[3], const double bc[6], int32_t *slot);

/* Release a grid's slot and storage (after the context's stream drains). */
int jac_pool_remove(jac_ctx *h, int32_t slot);

/* Bytes of the pool in use and its capacity, and the resident grids. */
int jac_pool_usage(jac_ctx *h, int64_t *used_bytes, int64_t *capacity_bytes, int32_t *grids);

/* ------------------------------------------------------------------ */
/* Server: continuous batching of solve requests                       */
/* ------------------------------------------------------------------ */

/* Solve requests (a grid, its boundary values and initial interior, a
 * residual tolerance and an iteration cap) are queued first come first
 * served and admitted while a slot (max_active) and room in an HBM budget
 * of budget_bytes are free. Every admitted grid stays resident until it
 * finishes. Each jac_server_step admits what fits, then advances every
 * resident grid by chunk_iters iterations in shared launches (one persistent
 * launch for the binary64 grids and one for the binary32 grids, on two
 * streams so they overlap) and reads every grid's binary64 residual: a grid
 * finishes after the first chunk whose residual is below its tolerance, or
 * when it reaches its cap. A grid's result therefore does not depend on
 * which other grids shared its launches. There is no counterpart of this
 * loop in the paper, which runs fixed iteration counts (Section IV-A). */
typedef struct jac_server jac_server;

typedef struct {
    int32_t running;       /* resident grids                              */
    int32_t queued;        /* requests waiting for admission              */
    int32_t finished_now;  /* grids retired by this step                  */
    int64_t cell_updates;  /* cell updates done since creation            */
    int64_t used_bytes;    /* bytes of the budget in use                  */
    int64_t budget_bytes;  /* the budget                                  */
} jac_server_stats_t;

typedef struct {
    int64_t id;
    int64_t iterations;    /* iterations run (a multiple of chunk_iters)  */
    double residual;       /* binary64 residual of the final state        */
    double t_submit;       /* seconds since the server was created        */
    double t_admit;
    double t_done;
    int32_t status;        /* JAC_OK, or the code that failed the request */
} jac_request_t;

int jac_server_create(jac_server **out, int64_t budget_bytes, int32_t max_active, int32_t bx, int32_t by,
                      int32_t bz, int32_t chunk_iters);
int jac_server_destroy(jac_server *s);

/* Queue a request; `init` (nx*ny*nz binary64 values, x fastest) is copied.
 * dtype JAC_F32 grids are stored and iterated in binary32 (values rounded
 * to nearest); their residual is still binary64. */
int jac_server_submit(jac_server *s, const int64_t dims[3], int32_t dtype, const double bc[6],
                      const double *init, double tol, int64_t max_iters, int64_t *req_id);

/* One admission + chunk + retirement round (synchronises). */
int jac_server_step(jac_server *s, jac_server_stats_t *stats);

/* Take one finished request's summary; JAC_ESTATE when none is waiting. */
int jac_server_poll(jac_server *s, jac_request_t *done);

/* Copy a finished request's final interior (binary64, x fastest; NULL to
 * discard it) and forget the request. */
int jac_server_result(jac_server *s, int64_t req_id, double *host_out, size_t n_cells);

/* Seconds since the server was created (the clock of jac_request_t). */
int jac_server_now(jac_server *s, double *seconds);

/* ------------------------------------------------------------------ */
/* Diagnostics                                                         */
/* ------------------------------------------------------------------ */

const char *jac_strerror(int code);
const char *jac_last_error(void);

/* Limit, in nanoseconds, of every device-side wait of the persistent mode
 * (default 2e9). After it the kernel records JAC_ETIMEOUT, stops issuing
 * work and returns; the context's next sync reports it. */
int jac_set_wait_limit_ns(jac_ctx *h, int64_t ns);

/* Test hook for the timeout path: while `block` >= 0, the persistent kernel
 * never publishes that block's progress counter after iteration
 * `after_iter`, so its neighbours' waits run out. -1 disables. */
int jac_debug_withhold_progress(jac_ctx *h, int32_t block, int64_t after_iter);

#ifdef __cplusplus
}
#endif

#endif /* JACOBI3D_H */
