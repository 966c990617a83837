/*
 * pyc.h -- C ABI of the run-time specialised map and map-reduce library for
 * GB300 (sm_103a).
 *
 * The operations follow Klockner et al., "GPU Scripting and Code Generation
 * with PyCUDA":
 *   - map (ElementwiseKernel, Sec. 3.2.4, Listing 3a): a C argument list plus a
 *     statement (or ';'-separated statements) executed for every value of the
 *     formal index i over arrays that all have the same length, in one pass
 *     with no temporaries;
 *   - map-reduce (ReductionKernel, Sec. 3.2.5, Listing 3b): a result type, a C
 *     argument list, a map expression in i, a reduce expression in the two
 *     formal values a and b, and an expression giving the neutral element;
 *     the result stays in device memory;
 *   - source is generated per specification, compiled at run time and cached
 *     by a hash of the source (Sec. 2, Fig. 1; Sec. 3.3 on run-time code
 *     generation and automated tuning);
 *   - launches are asynchronous on an optional stream (Sec. 3.1) and take a
 *     prepared argument layout (Sec. 3.1, prepared invocation).
 *
 * Conventions shared by every entry point:
 *   - Every call returns a pyc_status and never aborts.  On failure
 *     pyc_last_error() returns a message for the calling thread (for
 *     compile errors it contains the compiler log).
 *   - Device pointers are plain CUDA device addresses in the context that is
 *     current on the calling thread (the primary context of the device if no
 *     context is current).  The caller owns every buffer and stream passed in.
 *   - A stream argument is a CUstream / cudaStream_t; NULL is the legacy
 *     default stream.  Launches are enqueued and return immediately; device
 *     faults surface at the caller's next synchronisation.
 *   - Handles are safe to launch from several threads.  Creating a handle
 *     needs no GPU (parse, generate, compile); the first launch on a device
 *     loads the module there.  Handles may be created from several threads at
 *     once: a source that one thread is compiling is not compiled again by
 *     another, which waits for the first one's module (or its error).
 */
#ifndef PYC_H
#define PYC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PYC_VERSION_MAJOR 0
#define PYC_VERSION_MINOR 1

typedef struct CUstream_st* pyc_stream_t; /* same object as CUstream / cudaStream_t */
typedef struct pyc_map* pyc_map_t;
typedef struct pyc_reduce* pyc_reduce_t;

typedef enum {
  PYC_OK = 0,
  PYC_E_PARSE = 1,    /* malformed argument spec, statement or expression */
  PYC_E_COMPILE = 2,  /* run-time compilation failed; pyc_last_error() holds the log */
  PYC_E_ARG = 3,      /* invalid argument (null or misaligned pointer, bad size, ...) */
  PYC_E_CUDA = 4,     /* CUDA driver error, or no driver / device available */
  PYC_E_NOMEM = 5,    /* device or host allocation failed, or over a memory budget */
  PYC_E_BUSY = 6,     /* resource in use (e.g. a queue is full) */
  PYC_E_TIMEOUT = 7,  /* a bounded wait ran out */
  PYC_E_INTERNAL = 8, /* invariant violated inside the library */
  PYC_E_NOTFOUND = 9  /* unknown id */
} pyc_status;

/* Element / result types.  ARGMIN_F32 and ARGMAX_F32 are (value, index) pairs
 * laid out as pyc_argf32. */
typedef enum {
  PYC_F32 = 0,
  PYC_F64 = 1,
  PYC_BF16 = 2,
  PYC_F16 = 3,
  PYC_I32 = 4,
  PYC_I64 = 5,
  PYC_ARGMIN_F32 = 6,
  PYC_ARGMAX_F32 = 7,
  PYC_U8 = 8,
  PYC_I8 = 9,
  PYC_U32 = 10,
  PYC_U64 = 11,
  PYC_I16 = 12,
  PYC_U16 = 13
} pyc_dtype;

/* Result of an ARGMIN_F32 / ARGMAX_F32 reduction (16 bytes). */
typedef struct {
  float v;
  int32_t pad;
  int64_t i;
} pyc_argf32;

/* Creation options.  Zero in a tuning field means "use the tuned value for
 * the launch's size bucket, or the built-in default".  A NULL pyc_opts* means
 * all zero. */
typedef struct {
  int block;            /* threads per CTA: 0 or a multiple of 32 in [32, 512] */
  int vec_bytes;        /* bytes per vector access: 0, 16 or 32 */
  int items_per_thread; /* vector accesses per thread per tile (unroll): 0, 1, 2 or 4 */
  int compensated;      /* map-reduce only: 1 = compensated FP32 sum (two-sum per element,
                           pairwise (sum, error) combine, binary64 final combine).  Needs
                           result type F32 and reduce expression a+b. */
  int fmad;             /* 1 = let the compiler contract a*b+c into FMA.  0 (default) =
                           each +,-,* rounds as written, so results are reproducible
                           bit-for-bit against IEEE binary32 evaluation of the source. */
  const char* preamble; /* optional device code (helper functions, constants) placed
                           before the kernel; NULL = none */
  int debug_bounds;     /* 1 = bounds-checked build (a debugging aid, slower): every
                           array access the generated kernels make -- vector groups and
                           single elements, in single, batched, sharded and served
                           launches -- is checked against the array's index range and
                           its access width; the first violation is recorded and the
                           access skipped.  Read it with pyc_map_check_bounds /
                           pyc_reduce_check_bounds (scans: pyc_scan_sync).  Also
                           selected for every handle by $PYC_DEBUG_BOUNDS=1.  Accesses
                           a statement makes itself other than name[i] are not
                           checked. */
} pyc_opts;

/* Static description of one declared argument (for prepared invocation). */
typedef struct {
  const char* name;  /* owned by the handle */
  int is_pointer;    /* 1 = array (device pointer), 0 = scalar passed by value */
  int dtype;         /* pyc_dtype of the scalar or of the array element */
  int elem_bytes;    /* size of the scalar / array element */
  int scalar_offset; /* byte offset of a scalar inside the packed scalar block; -1 for arrays */
  int pointer_slot;  /* index into the ptrs[] array for arrays; -1 for scalars */
  int read;          /* array is read by the statement / map expression */
  int written;       /* array is written by the statement */
  int lifted;        /* array is only accessed as name[i], so it is moved through
                        registers with vector loads / stores */
} pyc_param_info;

/* ------------------------------------------------------------------ errors */

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next pyc_* call on the same thread. */
const char* pyc_last_error(void);

/* Library version string, e.g. "pyc 0.1 (sm_103a)". */
const char* pyc_version(void);

/* ------------------------------------------------------------------ map */

/* Create a map (ElementwiseKernel, Sec. 3.2.4, Listing 3a).
 *   argspec  C parameter list, e.g. "float a, float *x, float b, float *y, float *z".
 *            Types: float, double, int, unsigned, long long, unsigned long long,
 *            short, unsigned short, signed char, unsigned char, (u)int{8,16,32,64}_t,
 *            __nv_bfloat16 (bf16), __half (half).  bf16 / half storage is
 *            read and computed in binary32 and rounded to nearest even on store.
 *   stmt     statement(s) executed for each i in [0, n), e.g. "z[i] = a*x[i] + b*y[i]".
 *            i (long long) and n (long long) are in scope; names starting with
 *            "pyc_" are reserved.
 *   name     kernel name used in diagnostics (may be NULL).
 * On success *out owns the compiled module.  Errors: PYC_E_PARSE (spec or
 * statement), PYC_E_COMPILE (log in pyc_last_error()), PYC_E_ARG. */
pyc_status pyc_map_create(const char* argspec, const char* stmt, const char* name,
                          const pyc_opts* opts, pyc_map_t* out);

/* Launch a map over i in [0, n).
 *   ptrs     one device pointer per array parameter, in declaration order; every
 *            array must hold at least n elements.  Arrays may alias exactly (the
 *            same pointer, as in Listing 1's in-place a[i] *= 2); partial overlap
 *            is undefined.
 *   scalars  the scalar parameters packed in declaration order, each at its
 *            natural alignment (a C struct of the scalars; see pyc_param_info
 *            scalar_offset); may be NULL if there are none.
 *   stream   stream to enqueue on.
 * n == 0 is a no-op.  The kernel is launched with programmatic stream
 * serialization (Blackwell's dependent launch): it may be scheduled while the
 * previous kernel on the stream drains, but waits for that kernel to complete
 * before its first memory access, so ordering is the stream's and back-to-back
 * launches overlap their launch gaps.  pyc_reduce_launch likewise.  Errors:
 * PYC_E_ARG (n < 0, null or misaligned array), PYC_E_CUDA. */
pyc_status pyc_map_launch(pyc_map_t h, int64_t n, void* const* ptrs, const void* scalars,
                          pyc_stream_t stream);

/* Run a map on HOST arrays and return when the results are in host memory.
 * Every array must be accessed as name[i] alone (an elementwise statement),
 * else PYC_E_ARG.  host_ptrs: one host pointer per array.
 * If every array's n elements lie in page-locked host memory that the driver
 * maps into the device's address space at the same address (cuMemAllocHost,
 * cudaHostAlloc or registered memory, under unified addressing), the kernel runs
 * on the host arrays themselves: its loads and stores cross the chip-to-chip
 * link, with no staging copies.  Otherwise the arrays are streamed through
 * device staging buffers in chunks of 2^22 elements, overlapping host-to-device
 * copies, kernels and device-to-host copies on three streams of the library's
 * own: arrays the statement reads are copied in and arrays it writes are copied
 * back (one it may leave unwritten is also copied in); the staging buffers
 * (three chunks of every array) are allocated by the first staged call and kept
 * by the handle.  Synchronous: returns when the results are in host memory.
 * Errors as for pyc_map_launch. */
pyc_status pyc_map_launch_host(pyc_map_t h, int64_t n, void* const* host_ptrs,
                               const void* scalars);

/* For a handle created with opts.debug_bounds (the stand-in for a memory
 * checker, Sec. 3.1's automatic error checking carried into the kernels):
 * synchronise the current context, then read and clear the first out-of-range
 * or misaligned access recorded by the handle's kernels in that context since
 * the last call.  PYC_OK if there was none; PYC_E_INTERNAL naming the access
 * (kind, index or address, the range's end, block, thread) otherwise; PYC_E_ARG
 * for a handle built without the checks.  Test hook: $PYC_DEBUG_BOUNDS_SHRINK=k
 * at creation narrows every checked range by k elements at its top, so that a
 * test can make the checks fire without any access leaving its array (the
 * accesses they reject are skipped). */
pyc_status pyc_map_check_bounds(pyc_map_t h);
pyc_status pyc_reduce_check_bounds(pyc_reduce_t h);

/* Number of declared parameters and their descriptions. */
int pyc_map_num_params(pyc_map_t h);
pyc_status pyc_map_param(pyc_map_t h, int idx, pyc_param_info* info);
/* Size of the packed scalar block in bytes. */
int pyc_map_scalar_bytes(pyc_map_t h);
/* Generated CUDA source (owned by the handle). */
const char* pyc_map_source(pyc_map_t h);

/* Time the tuning candidates for n's size bucket on scratch buffers the library
 * allocates and frees (min(n, 2^28) elements per array, at most 6 GiB for all
 * arrays together, halved while the device cannot hold them), remember the
 * fastest for the handle and persist it in the tuning cache.  Synchronises the
 * stream.  (Automated tuning, Sec. 3.3.1.)  pyc_reduce_autotune and
 * pyc_scan_autotune size their scratch the same way.
 * With the environment variable PYC_AUTOTUNE=1, pyc_map_launch,
 * pyc_reduce_launch and pyc_scan_launch do this themselves: a launch at a size
 * bucket with no tuned configuration (none found in the tuning cache either)
 * runs with the default configuration and then tunes the bucket on its stream,
 * so that the launches after it use the tuned one -- unless the handle's options
 * fix the whole configuration, the stream is being captured, or another thread
 * is tuning the handle.  That launch allocates scratch and synchronises. */
pyc_status pyc_map_autotune(pyc_map_t h, int64_t n, pyc_stream_t stream);

/* The launch configuration (vector bytes, unroll, block) a launch of n
 * elements would use now: explicit options, else the tuned value of n's size
 * bucket, else the default. */
pyc_status pyc_map_config(pyc_map_t h, int64_t n, int* vec_bytes, int* unroll, int* block);

void pyc_map_destroy(pyc_map_t h);

/* ------------------------------------------------------------------ map-reduce */

/* Create a map-reduce (ReductionKernel, Sec. 3.2.5, Listing 3b).
 *   out_dtype    result type; the reduction accumulates in this type, except
 *                BF16/F16 results, which accumulate in binary32.
 *   neutral      C expression of the neutral element, e.g. "0" (Sec. 3.2.5);
 *                NULL for ARGMIN/ARGMAX selects (+-inf, INT64_MAX).
 *   reduce_expr  C expression in a and b (both of the accumulation type), e.g.
 *                "a+b"; must be associative and commutative.  NULL for
 *                ARGMIN/ARGMAX selects "smaller (larger) value, then smaller index".
 *   map_expr     C expression in i, e.g. "x[i]*y[i]"; NULL means "in[i]" for a
 *                single-array spec.  For ARGMIN/ARGMAX it gives the value; the
 *                index is i.
 *   argspec      C parameter list as for pyc_map_create.
 * Errors as for pyc_map_create. */
pyc_status pyc_reduce_create(pyc_dtype out_dtype, const char* neutral, const char* reduce_expr,
                             const char* map_expr, const char* argspec, const pyc_opts* opts,
                             pyc_reduce_t* out);

/* Reduce over i in [0, n) in one launch: every CTA folds its chunks, writes a
 * partial, and the last CTA to finish combines the partials and writes the
 * single result to d_out (one element of the result type).  No host round
 * trip.  n == 0 writes the neutral element.  Launches of one handle on one
 * stream are serialised by the stream; launches of one handle on different
 * streams use separate workspaces.  The result is a fixed function of
 * (n, tuning), independent of timing.  Errors as for pyc_map_launch. */
pyc_status pyc_reduce_launch(pyc_reduce_t h, int64_t n, void* const* ptrs, const void* scalars,
                             void* d_out, pyc_stream_t stream);

/* Sharded map-reduce: a range [0, n_total) cut into contiguous shards that live
 * on different devices (one process each), reduced with one exchange step.
 * Sec. 3.2.5 defines the reduction by an associative reduce expression and its
 * neutral element; together they make the reduction of the whole range equal
 * to the reduce expression applied, in shard order, to the reductions of the
 * shards (the paper itself runs on one device).
 *
 * pyc_reduce_shard folds shard [i0, i0 + n) into one accumulator record of
 * PYC_RECORD_BYTES (16) bytes at d_rec (device, 8-byte aligned):
 *   ptrs     one device pointer per array parameter, pointing at the shard's
 *            first element (global element i0); every array holds the shard's
 *            n elements.  The map expression sees the global index i in
 *            [i0, i0 + n) and n_total as n, so it may use i as a value and an
 *            ARGMIN / ARGMAX record carries the global index.  Every array must
 *            be accessed only as name[i] (else PYC_E_ARG): a shard holds no
 *            other elements.
 *   record   the shard's accumulator before its conversion to the result type:
 *            bytes [0, acc) hold the accumulation type (binary32 for F32, BF16
 *            and F16 results, the result type otherwise, pyc_argf32 for
 *            ARGMIN / ARGMAX), the rest are zero; for a compensated F32 handle,
 *            two binary64 values (hi, lo) whose sum is the shard's sum.  An empty
 *            shard (n == 0) gives the neutral element.
 * The launch, its chunk plan and its workspace are those of pyc_reduce_launch
 * for n elements; records on one stream are serialised by the stream.
 *
 * pyc_reduce_combine folds k >= 0 records (d_recs: k consecutive records in
 * shard order, device, 8-byte aligned) with the handle's reduce expression --
 * for a compensated handle, a binary64 (hi, lo) sum -- in record order and then
 * a fixed tree, converts once to the result type and writes one result to d_out
 * (device), as pyc_reduce_launch would.  k == 0 writes the neutral element.  One
 * launch of one CTA.  Integer sums, min / max and argmin / argmax give the same
 * bits as pyc_reduce_launch over the whole range; floating-point sums are
 * within the same bounds (another association order).  The exchange of
 * records between processes is the caller's, e.g. an all-gather of 16 bytes
 * per shard.
 * Errors: PYC_E_ARG (bad range, a non-elementwise array, NULL or misaligned
 * pointers), PYC_E_CUDA. */
#define PYC_RECORD_BYTES 16
pyc_status pyc_reduce_shard(pyc_reduce_t h, int64_t n_total, int64_t i0, int64_t n,
                            void* const* ptrs, const void* scalars, void* d_rec,
                            pyc_stream_t stream);
pyc_status pyc_reduce_combine(pyc_reduce_t h, int64_t k, const void* d_recs, void* d_out,
                              pyc_stream_t stream);

/* Segmented map-reduce: nseg independent reductions in one persistent launch.
 *   seg_offsets  HOST array of nseg+1 non-decreasing element offsets; segment s
 *                covers [seg_offsets[s], seg_offsets[s+1]) of every array.
 *   ptrs         base pointers of the concatenated arrays.
 *   d_out        nseg results (device).
 * The segment table is turned into a work list once (large segments split into
 * chunks, small ones packed one per warp); the list and the launch are cached
 * per (handle, table, pointers, scalars, output, stream) and replayed as a CUDA
 * graph on later calls with the same arguments.  Empty segments get the neutral
 * element.  Errors as for pyc_reduce_launch. */
pyc_status pyc_reduce_batched(pyc_reduce_t h, int64_t nseg, const int64_t* seg_offsets,
                              void* const* ptrs, const void* scalars, void* d_out,
                              pyc_stream_t stream);

/* Work plan of pyc_reduce_batched for a segment table, computed on the host
 * with no GPU work (introspection and tests; the launch builds the same plan).
 * Arguments as for pyc_reduce_batched (ptrs: the base arrays; they are not
 * dereferenced).  The plan has one task per segment: segments of at most 2048
 * elements first, in input order, reduced one warp each; then longer segments,
 * longest first (ties in input order), cut into chunks of whole tiles.
 *   task_info  NULL, or 6 int64 per task in plan order: segment index, length n,
 *              vector head (elements before the first aligned vector; -1 when
 *              the arrays share no alignment and the task runs element-wise),
 *              chunk length (elements), number of chunks (0 for one-warp tasks),
 *              first partial slot (used when it has more than one chunk).
 *   items      NULL, or 4 int32 per work item: (task, chunk, count, 0); chunk >= 0
 *              is one chunk of a long task (count 1); chunk = -1 is a bundle of
 *              `count` one-warp tasks starting at task index `task`.
 *   items_cap  capacity of items in work items (PYC_E_ARG if too small).
 *   n_items, n_slots  NULL, or the number of work items and of partial slots.
 * The configuration is the handle's batched one (pyc_reduce_batched_config).
 * Errors as for pyc_reduce_batched. */
pyc_status pyc_reduce_batched_plan(pyc_reduce_t h, int64_t nseg, const int64_t* seg_offsets,
                                   void* const* ptrs, const void* scalars, int64_t* task_info,
                                   int32_t* items, int64_t items_cap, int64_t* n_items,
                                   int64_t* n_slots);

/* Map-reduce launch that allocates nothing.  The paper has no counterpart.
 * For callers that cannot allocate device memory when they launch: programs
 * that reserve all device memory at start-up and must not allocate afterwards
 * (a fixed memory footprint), hosts whose device memory belongs to an outside
 * memory manager, and latency-critical loops where an allocation would
 * synchronise the device.  Arguments, kernel, chunk plan and result are those
 * of pyc_reduce_launch; the difference is where the per-CTA partials and the
 * finishing ticket live: in one static scratch area compiled into the library,
 * 65,792 bytes per GPU (4096 partial slots of up to 16 bytes, then the ticket),
 * which every GPU that loads the library holds until the process exits.  A
 * reduction whose chunk plan needs more partial bytes than that is rejected with
 * PYC_E_ARG (the planner caps a reduction at 4096 chunks, so none does today).
 * Set-up happens on first use and may allocate: the first call in a context
 * looks up the scratch address there (loading the library's own device module),
 * and the first call of each handle in each context loads that handle's kernels
 * and queries their occupancy.  So make one call of every handle you will use,
 * in every context you will use it in, before any stream capture and before the
 * point after which you may not allocate.  Later calls allocate nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.  All calls in a
 * context share its one scratch area, and it keeps what the last call left:
 * each call clears the ticket itself, but calls that overlap on the GPU (e.g. on
 * two streams with no ordering between them) race and give wrong results, so
 * serialise them.  Errors as for pyc_reduce_launch. */
pyc_status pyc_reduce_launch_static(pyc_reduce_t h, int64_t n, void* const* ptrs,
                                    const void* scalars, void* d_out, pyc_stream_t stream);

/* The static scratch area of pyc_reduce_launch_static in the current context
 * (the primary context of device $CUDA_DEVICE, default 0, if none is current):
 * *d_addr = its device address there, *bytes = its size (65,792).  Either
 * pointer may be NULL.  The first query in a context performs that context's
 * address lookup (the same one the launch's set-up does); no kernel runs.
 * Each context has its own area: the primary context and a context created
 * with cuCtxCreate on the same device get different addresses.  Like all of the
 * library's per-context state, entries are kept by context handle, so a context
 * the library has used must not be destroyed and replaced while the process
 * still calls the library.  Errors: PYC_E_ARG (both NULL), PYC_E_CUDA. */
pyc_status pyc_reduce_static_scratch(void** d_addr, int64_t* bytes);

/* Tune the batched launch (automated tuning, Sec. 3.3.1): time every vector
 * width x unroll x block candidate of the segmented reducer, and the
 * register-lean build of the 16-byte variants at each block, on this segment
 * table (same arguments as pyc_reduce_batched; d_out receives results), keep the
 * fastest for the handle's batched launches -- pyc_reduce_batched and the
 * server's map-reduce batches -- and persist it in the tuning cache.
 * Synchronises the stream. */
pyc_status pyc_reduce_batched_autotune(pyc_reduce_t h, int64_t nseg, const int64_t* seg_offsets,
                                       void* const* ptrs, const void* scalars, void* d_out,
                                       pyc_stream_t stream);

int pyc_reduce_num_params(pyc_reduce_t h);
pyc_status pyc_reduce_param(pyc_reduce_t h, int idx, pyc_param_info* info);
int pyc_reduce_scalar_bytes(pyc_reduce_t h);
/* Size in bytes of one result element (4, 8 or 16). */
int pyc_reduce_out_bytes(pyc_reduce_t h);
const char* pyc_reduce_source(pyc_reduce_t h);
pyc_status pyc_reduce_autotune(pyc_reduce_t h, int64_t n, pyc_stream_t stream);
pyc_status pyc_reduce_config(pyc_reduce_t h, int64_t n, int* vec_bytes, int* unroll, int* block);
/* Launch configuration (vector bytes, unroll, block size) of the handle's
 * batched launches (pyc_reduce_batched and the server's map-reduce batches):
 * the tuned one after pyc_reduce_batched_autotune, else the default, with any
 * fixed pyc_opts fields applied.  *reg_cap is 0 for the regular build of the
 * kernel, or the register cap of its register-lean build (16-byte variants: at
 * most 80 registers a thread, so more CTAs fit on an SM; one of the tuner's
 * candidates; a configuration fixed by pyc_opts fields is the regular build).  Any output pointer may be NULL.  Sec. 3.3.1 (the kept
 * variants).  PYC_E_ARG for a NULL handle. */
pyc_status pyc_reduce_batched_config(pyc_reduce_t h, int* vec_bytes, int* unroll, int* block,
                                     int* reg_cap);
void pyc_reduce_destroy(pyc_reduce_t h);

/* ------------------------------------------------------------------ scan */

/* Parallel prefix scan (Sec. 3.2.6: the packages' parallel prefix sums), in the
 * spec style of the map-reduce.
 *   dtype        value type: F32, F64, I32, I64, U32 or U64.
 *   neutral      C expression of the neutral element of scan_expr.
 *   scan_expr    associative C expression in a and b (a earlier, b later), e.g. "a+b".
 *   input_expr   value of element i, e.g. "x[i]".
 *   output_stmt  statement run for each i with `item` = the inclusive prefix
 *                scan_expr(input(0), ..., input(i)) and `prev_item` = the exclusive
 *                prefix (neutral for i = 0), e.g. "y[i] = item" or "y[i] = prev_item".
 *   argspec      C parameter list; "item" and "prev_item" are reserved names.
 * Floating-point association follows a fixed tree that depends on (n, tuning).
 * Errors as for pyc_reduce_create. */
typedef struct pyc_scan* pyc_scan_t;
pyc_status pyc_scan_create(pyc_dtype dtype, const char* neutral, const char* scan_expr,
                           const char* input_expr, const char* output_stmt, const char* argspec,
                           const pyc_opts* opts, pyc_scan_t* out);

/* Scan over i in [0, n): one launch on `stream`, no host round trip.  Tiles
 * of the index range are handed to CTAs in order; each tile finds its
 * exclusive prefix by looking back at the descriptors that earlier tiles
 * publish in the handle's workspace (one per (context, stream), grown on
 * demand; growing it synchronizes `stream`).  Each of those waits is bounded
 * (about a second of polling); if one runs out the launch still completes,
 * its output is not valid, and pyc_scan_sync reports PYC_E_TIMEOUT.  Aliasing
 * as for maps: output_stmt may write the array input_expr reads at the same
 * index (an in-place scan).  n == 0 is a no-op. */
pyc_status pyc_scan_launch(pyc_scan_t h, int64_t n, void* const* ptrs, const void* scalars,
                           pyc_stream_t stream);
/* Debugging aid: with the environment variable PYC_CHECK_BOUNDS=1 set when a
 * scan is created, its kernel checks every array and descriptor index and
 * records the first out-of-range one instead of accessing it; pyc_scan_sync
 * then fails with PYC_E_INTERNAL naming the index, tile and thread. */
/* Synchronizes `stream` and reports whether any scan launch of this handle on
 * it gave up a wait since the last call: PYC_OK, or PYC_E_TIMEOUT (the error
 * is then cleared and the workspace made ready for the next launch; launches
 * between the failing one and this call may have produced invalid output). */
pyc_status pyc_scan_sync(pyc_scan_t h, pyc_stream_t stream);
/* Test hook (the paper has no counterpart): pyc_scan_launch in which tile
 * `stall_tile` publishes no descriptor and every wait gives up after
 * `spin_limit` polls, so that the error path can be exercised without a fault.
 * stall_tile = -1 and spin_limit = 1 << 20 is pyc_scan_launch. */
pyc_status pyc_scan_launch_test(pyc_scan_t h, int64_t n, void* const* ptrs, const void* scalars,
                                pyc_stream_t stream, int64_t stall_tile, int64_t spin_limit);
int pyc_scan_num_params(pyc_scan_t h);
pyc_status pyc_scan_param(pyc_scan_t h, int idx, pyc_param_info* info);
int pyc_scan_scalar_bytes(pyc_scan_t h);
const char* pyc_scan_source(pyc_scan_t h);
pyc_status pyc_scan_autotune(pyc_scan_t h, int64_t n, pyc_stream_t stream);
/* (vec_bytes, unroll, block) a launch of n elements would use (as pyc_map_config). */
pyc_status pyc_scan_config(pyc_scan_t h, int64_t n, int* vec_bytes, int* unroll, int* block);
void pyc_scan_destroy(pyc_scan_t h);

/* ------------------------------------------------------------------ fused expressions */

/* Array arithmetic evaluated in one pass (Sec. 3.2.3-3.2.4: GPUArray operators
 * make one temporary per intermediate result; an ElementwiseKernel evaluates the
 * whole expression in a single pass).  The expression is compiled into one map
 * (or map-reduce) kernel, cached like any other spec.
 *
 * expr        prefix notation: a leaf or "(op operand ...)".  Leaves: $k (array
 *             argument k, element i), %k (scalar argument k), numeric literals
 *             (no suffix; a literal takes the type of the other operand, a
 *             fractional literal with integers gives double).
 *             Operators: + - * / min max pow (two operands), < <= > >= == !=
 *             (0 or 1, int), where (c, a, b: a if c != 0 else b), neg abs exp exp2
 *             log log2 sin cos tan tanh sqrt rsqrt floor ceil (one operand),
 *             casts f32 f64 i32 i64.
 * Typing      C-style: the wider of I32 < I64 < F32 < F64 (BF16 / F16 arrays read
 *             as F32); "/" and math functions of integers give F64; integer + - *
 *             wrap in two's complement.  Binary32 operations round each result
 *             (no contraction unless opts.fmad = 1); math functions are CUDA's.
 * args        nargs entries: arg_dtypes[k] (F32, F64, BF16, F16, I32, I64) and
 *             arg_is_array[k] (nonzero: an array of n elements).
 *
 * pyc_expr_map_create: the map "out[i] = expr" with argument list (a0 .. a{nargs-1},
 * out), out of out_dtype (F32, F64, BF16, F16, I32, I64).  Launch it with
 * pyc_map_launch: ptrs = the array arguments in order, then out; scalars packed
 * in argument order (pyc_map_param gives offsets).
 * pyc_expr_reduce_create: the map-reduce of expr with reduce "sum", "max" or
 * "min" into out_dtype (F32, F64, I32, I64); launch with pyc_reduce_launch (ptrs:
 * the arrays in order).
 * Errors: PYC_E_PARSE (syntax, unknown operator, operand count, an argument
 * used as the wrong kind), PYC_E_ARG (types), PYC_E_COMPILE. */
pyc_status pyc_expr_map_create(const char* expr, int nargs, const pyc_dtype* arg_dtypes,
                               const int* arg_is_array, pyc_dtype out_dtype,
                               const pyc_opts* opts, pyc_map_t* out);
pyc_status pyc_expr_reduce_create(const char* expr, int nargs, const pyc_dtype* arg_dtypes,
                                  const int* arg_is_array, pyc_dtype out_dtype,
                                  const char* reduce, const pyc_opts* opts, pyc_reduce_t* out);
/* The type of expr under the rules above (F32, F64, I32 or I64) in *out. */
pyc_status pyc_expr_type(const char* expr, int nargs, const pyc_dtype* arg_dtypes,
                         const int* arg_is_array, pyc_dtype* out);

/* ------------------------------------------------------------------ memory pools */

/* Memory pools (Sec. 3.2.6: allocation calls are expensive, so blocks that a
 * program frees are retained and handed out again for later requests of a
 * similar size; pools exist for device and for page-locked host memory).
 * Requests are rounded up to a size class: 512 bytes, or 8 classes per power
 * of two above (at most 1/8 of a block unused); a block is reused only for its
 * own class.  Reuse is stream-ordered: a block freed with stream s is handed out
 * at once for a request on s, and for requests on other streams once the work
 * queued on s before the free has finished (an event recorded at the free).
 * The pool is thread-safe.  Retained blocks return to the system on
 * pyc_pool_trim, on destroy, when retained bytes pass max_retained, and when a
 * system allocation fails (the allocation is then retried once). */
typedef struct pyc_pool* pyc_pool_t;
typedef enum {
  PYC_POOL_DEVICE = 0, /* cuMemAlloc: device memory of the current context's device */
  PYC_POOL_PINNED = 1, /* cuMemAllocHost: page-locked host memory */
  PYC_POOL_HOST = 2    /* ordinary host memory (aligned_alloc); streams are ignored */
} pyc_pool_kind;
typedef struct {
  int64_t max_bytes;    /* cap on bytes taken from the system (live + retained); 0 = none */
  int64_t max_retained; /* cap on retained (freed, unreturned) bytes; 0 = none */
} pyc_pool_cfg;
typedef struct {
  int64_t live_bytes, live_blocks;         /* handed out and not yet freed */
  int64_t retained_bytes, retained_blocks; /* freed, kept for reuse */
  int64_t system_bytes;                    /* live + retained */
  int64_t hits, misses;                    /* requests served by reuse / by the system */
  int64_t system_allocs, system_frees;
} pyc_pool_stats;
/* The size class (bytes actually reserved) of a request of `bytes`. */
int64_t pyc_pool_block_size(int64_t bytes);
/* cfg may be NULL (no limits).  Device and pinned pools use the current context
 * (the primary context of device $CUDA_DEVICE, default 0, if none is current). */
pyc_status pyc_pool_create(pyc_pool_kind kind, const pyc_pool_cfg* cfg, pyc_pool_t* out);
/* *ptr = a block of at least `bytes` (> 0), 256-byte aligned, to be used first on
 * `stream`.  PYC_E_NOMEM when the system (or max_bytes) cannot supply it. */
pyc_status pyc_pool_alloc(pyc_pool_t p, int64_t bytes, pyc_stream_t stream, void** ptr);
/* Return a block; `stream` is the last stream that uses it (work already queued
 * there may still be running).  NULL ptr is a no-op; a pointer this pool did not
 * hand out (or one freed twice) is PYC_E_ARG. */
pyc_status pyc_pool_free(pyc_pool_t p, void* ptr, pyc_stream_t stream);
/* Return every retained block to the system (waiting for the work that used it). */
pyc_status pyc_pool_trim(pyc_pool_t p);
pyc_status pyc_pool_get_stats(pyc_pool_t p, pyc_pool_stats* stats);
/* Returns retained AND live blocks to the system: live blocks become invalid. */
void pyc_pool_destroy(pyc_pool_t p);

/* ------------------------------------------------------------------ sparse matrices, CG */

/* Sparse matrices and a conjugate-gradient solver (Sec. 3.2.6: GPU sparse
 * matrices following Bell and Garland's SpMV, and a CG-based Krylov solver for
 * large sparse linear systems).
 *
 * pyc_csr_create wraps a CSR matrix already in device memory (the caller owns it
 * and keeps it alive): rowptr int64[nrows + 1] (rowptr[0] = 0, nondecreasing,
 * rowptr[nrows] = nnz), colidx int32[nnz] (each < ncols < 2^31), vals[nnz] of vt
 * (F32 or F64).  Every array, here and in the calls below, must be aligned to
 * its element size, and x, y, b must not be NULL (else PYC_E_ARG).  Indices are
 * not checked: out-of-range ones are undefined behaviour.  The handle compiles its kernels (cached) and picks T, the lanes per
 * row, from the mean row length. */
typedef struct pyc_csr* pyc_csr_t;
pyc_status pyc_csr_create(int64_t nrows, int64_t ncols, int64_t nnz, const void* rowptr,
                          const void* colidx, const void* vals, pyc_dtype vt, pyc_csr_t* out);
/* The width the matrix-vector product uses; set it.  1, 2, 4, ..., 32: lanes per
 * row over the CSR arrays.  0: a sliced-ELL copy that the handle builds from the
 * CSR arrays when width 0 is set (or tried by pyc_spmv_autotune, when padding
 * would at most double the stored entries): rows in slices
 * of 32, each slice padded to its longest row and stored entry-major, so that a
 * warp reads its rows' entries in 128-byte pieces and no row pointers; row
 * lengths of 1, 2 or 4 bytes.  Each row is still added in entry order (the same
 * bits as one lane per row).  The copy is a snapshot: later changes to the
 * caller's arrays are seen after width 0 is set again.  Setting width 0 runs on
 * the legacy default stream and returns when the copy is built; another width
 * frees the copy. */
pyc_status pyc_csr_width(pyc_csr_t a, int* width);
pyc_status pyc_csr_set_width(pyc_csr_t a, int width);
/* y = A x on `stream` (x: ncols, y: nrows elements of vt, device; x and y must not
 * overlap).  Each row is folded per lane, then across its lanes in a fixed tree. */
pyc_status pyc_spmv(pyc_csr_t a, const void* x, void* y, pyc_stream_t stream);
/* Time every width on (x, y) and keep the fastest for this matrix (building the
 * sliced copy to try width 0, and freeing it if another width wins). */
pyc_status pyc_spmv_autotune(pyc_csr_t a, const void* x, void* y, pyc_stream_t stream);

typedef struct {
  int64_t iterations; /* CG steps taken */
  double residual;    /* ||r|| / ||b|| at exit (the recurrence's r; ||r|| if b = 0) */
  int converged;      /* residual <= rtol */
  int pad;
} pyc_cg_info;
/* Solve A x = b for symmetric positive definite A by conjugate gradients
 * (Hestenes-Stiefel): x holds the initial guess on entry and the solution on
 * exit (device, nrows elements; b likewise).  Stops when ||r|| <= rtol ||b|| or
 * after maxit steps.  Runs on `stream`: steps are queued as CUDA graphs of 8
 * (re-captured when x, the width, the sliced copy or the work space change) with two
 * groups in flight while the host tests the previous group's residual; steps
 * queued past convergence change nothing.  The handle keeps 3 vectors of work
 * space per (context, stream); one solve at a time per (handle, stream).  A
 * breakdown (p.Ap = 0 before convergence) stops progress; the result then
 * reports converged = 0.  While it runs, the work vectors (and x) that fit
 * together in 9/16 of L2 are held there with an evict-last cache policy and the
 * matrix is read evict-first; at exit their L2 lines return to normal priority.
 * The width in use (lanes per row or the sliced copy) is the handle's. */
pyc_status pyc_cg_solve(pyc_csr_t a, const void* b, void* x, double rtol, int64_t maxit,
                        pyc_stream_t stream, pyc_cg_info* info);
void pyc_csr_destroy(pyc_csr_t a);

/* ------------------------------------------------------------------ serving */

/* A request-serving loop over map and map-reduce handles (continuous
 * batching).  Not in the paper: it serves many independent map / map-reduce
 * requests of different sizes that arrive over time.  A scheduler thread
 * admits queued requests in arrival order while the logical bytes of admitted,
 * unreleased requests (every array of the request, n elements each, plus the
 * result) stay within mem_budget_bytes; groups admitted requests by handle into
 * one batched launch each (a request is cut into about 256 chunks of at least
 * 4096 elements and at most 2^16, both rounded up to whole tiles, one CTA each;
 * a reduction of at most 2048 elements takes one warp); spreads the batches
 * over num_streams streams, at
 * most max_inflight at a time; and retires them by completion events.  A
 * request's result depends only on the request itself, never on the other
 * requests of its batch.  The server owns a device arena (arena_bytes) for map
 * outputs it allocates: a written-only array of a map request may be passed as
 * NULL and is then allocated from the arena (returned in pyc_result.d_out) and
 * kept until pyc_server_release.  It starts at the address of the request's
 * first given array modulo 256 (rounded down to its element size), so that all
 * of the request's arrays can take the vector path together. */
typedef struct pyc_server* pyc_server_t;

#define PYC_REQ_MAP 0
#define PYC_REQ_REDUCE 1

typedef struct {
  int64_t mem_budget_bytes; /* admission cap in bytes (> 0) */
  int64_t arena_bytes;      /* device arena for server-allocated outputs; 0 = min(budget, 8 GiB) */
  int num_streams;          /* 0 = 4 (at most 64) */
  int max_batch;            /* requests per batched launch; 0 = 256 (at most 4096) */
  int max_inflight;         /* launched, unfinished batches; 0 = 8 (at most 256) */
  int max_queue;            /* waiting requests before submit answers PYC_E_BUSY; 0 = 2^20 */
} pyc_server_cfg;

typedef struct {
  int kind;             /* PYC_REQ_MAP or PYC_REQ_REDUCE */
  int pad;
  void* handle;         /* pyc_map_t or pyc_reduce_t; must outlive the request */
  int64_t n;            /* elements, 0 <= n <= 2^34 */
  void* const* ptrs;    /* device arrays in declaration order (copied at submit) */
  const void* scalars;  /* packed scalars as for the launch calls (copied at submit) */
  int64_t deadline_us;  /* > 0: fail with PYC_E_TIMEOUT if not admitted within this time */
} pyc_request;

typedef struct {
  int status;           /* PYC_OK, or why the request failed */
  int batch_size;       /* requests in the launch that ran it */
  void* d_out;          /* map: first server-allocated output (NULL if none) */
  unsigned char value[16];  /* map-reduce: the result, pyc_reduce_out_bytes bytes */
  int64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns; /* steady clock; done = completion seen */
} pyc_result;

typedef struct {
  int64_t submitted, completed, failed, batches;
  int64_t admitted_bytes;      /* current logical bytes of admitted, unreleased requests */
  int64_t peak_admitted_bytes; /* never above mem_budget_bytes */
  int64_t queued;              /* waiting for admission */
  int64_t arena_in_use;        /* bytes of server-allocated outputs */
} pyc_server_stats;

/* Create a server on the current context (allocates its streams, arena and
 * per-batch slots: 16 MiB device + 16 MiB pinned host each).  Errors:
 * PYC_E_ARG, PYC_E_CUDA, PYC_E_NOMEM. */
pyc_status pyc_server_create(const pyc_server_cfg* cfg, pyc_server_t* out);

/* Queue a request; *id identifies it until pyc_server_release.  Errors:
 * PYC_E_ARG (bad request: among others a NULL array other than a written-only
 * map output, or an array not aligned to its element size; checked here, so a
 * bad request never joins a batch), PYC_E_NOMEM (larger than the whole budget),
 * PYC_E_BUSY (queue full or shutting down). */
pyc_status pyc_server_submit(pyc_server_t s, const pyc_request* req, uint64_t* id);

/* Wait up to timeout_us (0 = do not wait) for request id to finish.  PYC_OK
 * fills *res (res->status says whether the request succeeded); PYC_E_TIMEOUT
 * if it is still running; PYC_E_NOTFOUND for an unknown id. */
pyc_status pyc_server_poll(pyc_server_t s, uint64_t id, pyc_result* res, int64_t timeout_us);

/* Forget a finished request: frees its server-allocated outputs and returns its
 * bytes to the budget.  PYC_E_BUSY if it has not finished. */
pyc_status pyc_server_release(pyc_server_t s, uint64_t id);

pyc_status pyc_server_get_stats(pyc_server_t s, pyc_server_stats* st);

/* Fail queued requests, wait for launched batches, free everything. */
void pyc_server_destroy(pyc_server_t s);

/* Test hook (the paper has no counterpart): a serving loop whose batches run
 * on the host, so that everything in it but the device work -- admission
 * against the budget in arrival order, grouping by handle, batch slots and the
 * in-flight limit, deadlines, queue limits, outputs allocated by the server
 * (from a host arena here), release, replay -- runs and can be tested without
 * a GPU.  Each launched batch is handed to one executor thread, which calls
 * `exec` once per request in batch order with the request as submitted except
 * `ptrs`, which holds the arrays with the server's outputs filled in; for a
 * map-reduce, exec writes the result (pyc_reduce_out_bytes bytes) to `value`.
 * Its return value becomes the request's status (PYC_OK = 0).  The batch is
 * retired when every call has returned.  cfg as for pyc_server_create (a
 * default arena of at most 256 MiB of host memory); PYC_REPLAY_DIRECT is not
 * available.  Handles may be created without a GPU (run-time compilation needs
 * none).  Errors: PYC_E_ARG. */
typedef int (*pyc_host_exec_fn)(void* user, const pyc_request* req, void* value);
pyc_status pyc_server_create_host(const pyc_server_cfg* cfg, pyc_host_exec_fn exec, void* user,
                                  pyc_server_t* out);

/* Trace replay for load measurement.  Submits reqs[k] at t0 + arrival_ns[k]
 * (an open loop; all at t0 when arrival_ns is NULL), collects and releases every
 * request as it finishes and stores its pyc_result in results[k], with
 * t_submit_ns set to the request's arrival time.  mode PYC_REPLAY_SERVER goes
 * through the serving loop; PYC_REPLAY_DIRECT is the per-request baseline: each
 * request launched alone as it arrives with pyc_map_launch / pyc_reduce_launch
 * kernels on one stream.  Returns when every request has finished. */
#define PYC_REPLAY_SERVER 0
#define PYC_REPLAY_DIRECT 1
pyc_status pyc_server_replay(pyc_server_t s, int64_t nreq, const pyc_request* reqs,
                             const int64_t* arrival_ns, int mode, pyc_result* results);

/* ------------------------------------------------------------------ fault injection */

/* Test hook (the paper has no counterpart; it stands in for failures that tests
 * cannot cause on a shared GPU): make the library's own host-side steps fail on
 * purpose, so that its error paths run -- Sec. 3.1's rule that every failure
 * surfaces as an error, never as a crash or a silent wrong result.
 *   PYC_INJECT_ALLOC     the next `value` system allocations the library makes
 *                        (device cuMemAlloc, page-locked cuMemAllocHost, host-pool
 *                        blocks) fail as the driver does when memory runs out:
 *                        callers see PYC_E_NOMEM (a pool first returns its
 *                        retained blocks and retries once).
 *   PYC_INJECT_COMPILE   the next `value` run-time compilations fail with
 *                        PYC_E_COMPILE (cache hits do not compile).
 *   PYC_INJECT_STALL_MS  the next serving-loop scheduler to wake sleeps `value` ms
 *                        before admitting requests (a late scheduler: deadlines
 *                        run out, PYC_E_TIMEOUT).
 *   PYC_INJECT_ADMIT     the next `value` requests a serving loop comes to admit
 *                        are rejected there, as one the budget can never hold:
 *                        the request fails with PYC_E_NOMEM, those behind it
 *                        are admitted as usual.
 * value = 0 clears the kind.  Nothing is injected into the GPU.  Process-wide;
 * not for production use.  Errors: PYC_E_ARG (unknown kind, value < 0). */
typedef enum {
  PYC_INJECT_ALLOC = 0,
  PYC_INJECT_COMPILE = 1,
  PYC_INJECT_STALL_MS = 2,
  PYC_INJECT_ADMIT = 3
} pyc_inject_kind;
pyc_status pyc_test_inject(pyc_inject_kind what, int64_t value);

/* ------------------------------------------------------------------ cache */

/* Kernel cache statistics since process start: compiled = NVRTC compilations,
 * disk_hits = modules read from the on-disk cache, mem_hits = in-memory hits.
 * The on-disk cache lives in $PYC_CACHE_DIR (default $HOME/.cache/pyc).  With
 * the environment variable PYC_LOG=1 the library writes one line to stderr for
 * each compilation (with its time), disk-cache load, tuning result, segmented
 * plan and server creation or destruction. */
void pyc_cache_stats(int64_t* compiled, int64_t* disk_hits, int64_t* mem_hits);

#ifdef __cplusplus
}
#endif
#endif /* PYC_H */
