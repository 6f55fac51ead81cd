/*
 * hdarray.h -- C ABI of the GB300 HDArray library (libhdarray.so).
 *
 * An HDArray is an array split over logical devices ("partitions").  Each logical device owns a
 * device buffer of its own in the GPU's memory.  Every HDArrayApplyKernel call first computes,
 * from the kernel's use/def sections and the array's GDEF bookkeeping, exactly which array
 * sections each device must receive from which other device (Eq. 1-2 of Cho, Kwon & Midkiff,
 * "HDArray", Sec. 2.2), moves them between the device buffers with the library's own copy kernels
 * (or inside the stencil kernel itself), runs the kernel on every device's work region, and
 * updates the bookkeeping (Eq. 3-4).  The paper's MPI messages and host-staged rectangle copies
 * become on-GPU section copies between buffers.
 *
 * Conventions for every call below:
 *   - Coordinates are up to three dimensions, dimension 0 outermost (row-major).  Sizes and
 *     bounds are int64_t.  Boxes are half-open [lo, hi); trapezoid corners name elements.
 *   - Pointers named uA / res are host pointers or device pointers (any pointer the CUDA runtime
 *     can address); the library never keeps them after the call returns.
 *   - Calls of the paper's prototypes that return void record an error code readable with
 *     HDArrayGetLastError(); every other call returns it: 0 = HDARRAY_OK, negative = error.
 *     Nothing aborts the process.
 *   - The library runs on the CUDA device that is current at HDArrayInit, on one stream
 *     (HDArraySetStream); keep that device current while calling it.  Kernel launches are
 *     asynchronous; HDArrayRead, HDArrayReduce and HDArraySync wait for the stream.
 *   - Not thread safe: one host thread drives the library.
 */
#ifndef HDARRAY_H
#define HDARRAY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------------------------------- */
/* Types and codes                                                                            */
/* ---------------------------------------------------------------------------------------- */

/* Opaque handle of an HDArray (Sec. 3.1, HDArrayCreate).  Owned by the library; freed by
 * HDArrayFree or HDArrayExit. */
typedef struct HDArray HDArray_t;

/* Partition types of HDArrayPartition (Sec. 3.1): ROW splits dimension 0, COL dimension 1, BLOCK
 * dimensions 0 and 1 on a Pr x Pc device grid (Pr the largest divisor of P with Pr*Pr <= P,
 * devices in row-major grid order).  Even split: the first (n mod P) parts get one extra row. */
typedef enum { HDARRAY_ROW = 0, HDARRAY_COL = 1, HDARRAY_BLOCK = 2 } PART_T;

/* Reduction operators of HDArrayReduce (Sec. 3.1, Table 2). */
typedef enum { HDARRAY_SUM = 0, HDARRAY_PROD = 1, HDARRAY_MAX = 2, HDARRAY_MIN = 3 } REDUCE_OP;

#ifdef HDARRAY_SHORT_NAMES /* the paper's spellings, opt-in because they collide easily */
#define ROW HDARRAY_ROW
#define COL HDARRAY_COL
#define BLOCK HDARRAY_BLOCK
#define SUM HDARRAY_SUM
#define PROD HDARRAY_PROD
#define MAX HDARRAY_MAX
#define MIN HDARRAY_MIN
#endif

#define HDARRAY_OK 0
#define HDARRAY_ERR_INVAL (-1)       /* bad argument, unknown name, wrong type or shape        */
#define HDARRAY_ERR_NOMEM (-2)       /* a host or device allocation failed                      */
#define HDARRAY_ERR_RACE (-3)        /* two devices define the same element in one call         */
#define HDARRAY_ERR_RANGE (-4)       /* a section lies outside its array                        */
#define HDARRAY_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                      */
#define HDARRAY_ERR_CUDA (-6)        /* a CUDA call failed (no device, launch failure ...)      */
#define HDARRAY_ERR_STATE (-7)       /* not initialised, stale graph, batch misuse ...          */
#define HDARRAY_ERR_UNSUPPORTED (-8) /* valid request this build does not implement            */

/* The '*' offset component (Sec. 3, offset clauses): every element of that dimension. */
#define HDARRAY_ALL INT32_MIN

/* Execution forms (HDArraySetMode). */
#define HDARRAY_MODE_FUSED 0 /* exchange fused into the kernel, all devices in one launch     */
#define HDARRAY_MODE_PLAIN 1 /* one copy launch per section, one kernel launch per device     */

/* HDArrayInitEx flags. */
#define HDARRAY_INIT_HOST_ONLY 1u /* bookkeeping only: no GPU, no buffers, no kernel launches */

/* ---------------------------------------------------------------------------------------- */
/* The paper's calls (Sec. 3.1, Table 2)                                                      */
/* ---------------------------------------------------------------------------------------- */

/* HDArrayInit (Table 2): initialise the runtime on the current CUDA device and return the
 * device ID (0).  argc/argv and kpath are accepted and ignored (the kernels are built into
 * the library).  dpath may name a text file whose first
 * token is the default number of logical devices used by HDArrayPartition; NULL means the
 * environment variable HDARRAY_NDEV, else 1.  Returns < 0 on error. */
int HDArrayInit(int argc, char *argv[], const char *kpath, const char *dpath);

/* HDArrayExit (Table 2): free every HDArray, partition, plan, graph and device buffer. */
void HDArrayExit(void);

/* HDArrayShowDeviceInfo (Table 2): print the CUDA device's name, SM count and memory. */
void HDArrayShowDeviceInfo(int devID);

/* HDArrayCreate (Table 2): a new HDArray named sym with element type "double", "float" or
 * "bf16" (bfloat16 bit patterns, 2 bytes) and dim (1..3) sizes passed as int varargs.  Device
 * buffers are allocated lazily, per logical device, covering what that device touches, and are
 * zero-filled; nothing is copied from uA (which may be NULL).  Returns NULL on error. */
HDArray_t *HDArrayCreate(const char *sym, const char *type, void *uA, int dim, ...);

/* HDArrayPartition (Table 2): even partition of a work region over the default number of
 * logical devices.  Varargs (int): sizes[dim], then lo[dim], then hi[dim] of the region
 * (half-open), as in HDArrayPartition(ROW, 2, ni, nj, 0, 0, ni, nj) of Listing 2.  Returns the
 * partition ID (>= 0) or < 0 on error. */
int HDArrayPartition(PART_T type, int dim, ...);

/* HDArrayApplyKernel (Table 2, Sec. 3.1): exchange, then run kernel kName on every logical
 * device's work region of partition partID, then update GDEF.  Varargs: the kernel's
 * arguments in its declared order; HDArray_t* for array arguments, double for floating scalars
 * (a float argument is promoted to double by the C varargs rules), int for integer scalars.
 * Built-in kernels and their arguments:
 *   "jacobi2d"  (HDArray_t *X, HDArray_t *Y)               Y = 4-neighbour mean of X (Sec. 5)
 *   "copy"      (HDArray_t *X, HDArray_t *Y)               Y = X          (Sec. 5, kernel 2)
 *   "stencil3d" (HDArray_t *X, HDArray_t *Y)               Y = 6-neighbour mean of X (3-D)
 *   "conv2d"    (HDArray_t *X, HDArray_t *Y, double w0 .. w8)  Y = 3 x 3 convolution of X
 *               (Sec. 5, eight neighbours): Y[i][j] = sum_{a,b=0..2} w[3a+b] X[i+a-1][j+b-1],
 *               summed in that order, each product rounded, in X's arithmetic precision
 *   "sqdiff"    (HDArray_t *X, HDArray_t *Y, HDArray_t *R) R = (X - Y)^2 in double
 *   "gemm"      (A, B, C, double alpha, double beta, int ni, int nj, int nk)   (Listing 3)
 *   "trmm"      (A, B, C, double alpha, double beta)       the same with A lower triangular
 *   "exchange"  (HDArray_t *X)                             the communication step alone
 * Asynchronous on the library stream. */
void HDArrayApplyKernel(const char *kName, int partID, ...);

/* HDArrayRead (Table 2): copy every logical device's region of partition partID from the
 * HDArray into the user array uA (full-size, row-major, the array's element type).  Each device
 * first receives the elements of its region it does not hold.  Synchronous. */
void HDArrayRead(HDArray_t *hA, void *uA, int partID);

/* HDArrayWrite (Table 2): copy every logical device's region of partition partID from the user
 * array uA (full-size, row-major) into that device's buffer.  This is a definition by each
 * device of its region (it becomes the owner; other copies become stale).  Overlapping regions
 * are a race.  From pinned (page-locked) host memory into buffers that already cover the regions,
 * the copies run on the library's own copy stream, after the library's last work on hA and
 * alongside its work on other arrays; everything the library later does with hA waits for them.
 * Keep uA unchanged until a synchronising call (Read, Reduce, Sync) has returned.  From pageable
 * host memory the call returns once uA has been read; device pointers are copied on the library
 * stream.  HDARRAY_ASYNC_WRITE=0 puts every copy on the library stream. */
void HDArrayWrite(HDArray_t *hA, void *uA, int partID);

/* HDArrayReduce (Table 2): reduce the regions of partition partID (each element once) to one
 * scalar of the array's element type at *res (host pointer), accumulating in double.  Each
 * device first receives what it does not hold of its region.  Synchronous. */
void HDArrayReduce(HDArray_t *hA, void *res, REDUCE_OP op, int partID);

/* HDArraySetAbsoluteUse / Def (Table 2, Sec. 3 "use@/def@"): add the box lo[dim], hi[dim]
 * (int varargs, half-open) to LUSE (LDEF) of logical device devID for array hA in kernel kName
 * with partition partID.  Once any box is set for (kName, partID, hA), that array's offsets are
 * bypassed for that kernel and partition; devices without boxes use (define) nothing. */
void HDArraySetAbsoluteUse(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...);
void HDArraySetAbsoluteDef(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...);

/* HDArraySetTrapezoidUse / Def (Table 2, Sec. 3.1): add a 2-D trapezoid to LUSE (LDEF), given by
 * its upper-left, upper-right, lower-left and lower-right corner elements as 8 int varargs
 * (row, col each).  The top edge is the upper corners' row, the bottom edge the lower corners'
 * row; row r spans, inclusively, the columns between the two edge lines, each rounded down in
 * exact integer arithmetic.  dim must be 2. */
void HDArraySetTrapezoidUse(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...);
void HDArraySetTrapezoidDef(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...);

/* ---------------------------------------------------------------------------------------- */
/* Non-variadic forms (same meaning; return 0 or a negative error code)                      */
/* ---------------------------------------------------------------------------------------- */

/* Initialise with ndev default logical devices.  flags: HDARRAY_INIT_HOST_ONLY keeps the
 * bookkeeping (partitions, sections, GDEF, plans) but touches no GPU: no buffers are allocated,
 * nothing is launched, data calls move no data.  Used to inspect communication on any host. */
int HDArrayInitEx(int ndev, unsigned flags);

HDArray_t *HDArrayCreatev(const char *sym, const char *type, void *uA, int dim,
                          const int64_t *sizes);

/* nparts = 0 uses the default device count.  sizes/lo/hi: dim values each. */
int HDArrayPartitionv(PART_T type, int nparts, int dim, const int64_t *sizes, const int64_t *lo,
                      const int64_t *hi);

/* The partition clause (Sec. 3, Listing 1): explicit work boxes, one per logical device;
 * lo and hi hold nparts * dim values (device-major).  A device with an empty box gets no work.
 * Returns the partition ID. */
int HDArrayPartitionManual(int dim, const int64_t *sizes, int nparts, const int64_t *lo,
                           const int64_t *hi);

/* ApplyKernel with nargs array handles and nscal scalars (all as double, integers included). */
int HDArrayApplyKernelv(const char *kName, int partID, int narr, HDArray_t *const *arrs,
                        int nscal, const double *scal);

int HDArrayReadv(HDArray_t *hA, void *uA, int partID);
int HDArrayWritev(HDArray_t *hA, const void *uA, int partID);
int HDArrayReducev(HDArray_t *hA, void *res, REDUCE_OP op, int partID);

/* HDArrayReduce returning the double accumulator itself (element type irrelevant). */
int HDArrayReduceD(HDArray_t *hA, double *res, REDUCE_OP op, int partID);

int HDArraySetAbsoluteUsev(const char *kName, int partID, HDArray_t *hA, int devID, int dim,
                           const int64_t *lo, const int64_t *hi);
int HDArraySetAbsoluteDefv(const char *kName, int partID, HDArray_t *hA, int devID, int dim,
                           const int64_t *lo, const int64_t *hi);
/* corners: ul_r, ul_c, ur_r, ur_c, ll_r, ll_c, lr_r, lr_c. */
int HDArraySetTrapezoidUsev(const char *kName, int partID, HDArray_t *hA, int devID,
                            const int64_t *corners);
int HDArraySetTrapezoidDefv(const char *kName, int partID, HDArray_t *hA, int devID,
                            const int64_t *corners);

/* ---------------------------------------------------------------------------------------- */
/* Extensions (no counterpart call in the paper; each stands in for something the paper does */
/* outside its library API)                                                                   */
/* ---------------------------------------------------------------------------------------- */

/* Replace the use (def) offsets of argument argIndex of kernel kName: noff offsets of 3 int32
 * each (unused dimensions 0; HDARRAY_ALL for '*').  Stands in for the use/def pragma clauses
 * (Sec. 3, Table 1), which the paper's frontend compiles into the runtime's kernel table. */
int HDArraySetOffsetUse(const char *kName, int argIndex, int noff, const int32_t *offs);
int HDArraySetOffsetDef(const char *kName, int argIndex, int noff, const int32_t *offs);

/* Free one HDArray and its device buffers. */
int HDArrayFree(HDArray_t *hA);

/* Number of default logical devices (HDArrayInit). */
int HDArrayNumDevices(void);

/* Run all following work on this cudaStream_t (NULL: the library's own non-blocking stream). */
int HDArraySetStream(void *stream);

/* HDARRAY_MODE_FUSED (default) or HDARRAY_MODE_PLAIN. */
int HDArraySetMode(int mode);

/* Precision form of binary32 GEMMs (gemm, trmm, syrk) on the tensor cores, after Henry, Tang &
 * Heinecke (ARITH 2019): HDARRAY_GEMM_BF16X3 (default) splits every operand value into two
 * bfloat16 parts and keeps three products per pair (about 3 * 2^-16 of |a||b| per product);
 * HDARRAY_GEMM_BF16X6 splits into three parts and keeps six products (about 2^-22), as accurate
 * as binary32 products, at twice the tensor work.  Plans compiled for the other form are
 * recompiled on their next call; graphs recorded before keep the form they recorded.  Returns
 * HDARRAY_ERR_INVAL for another value, HDARRAY_ERR_STATE inside a batch or a graph recording. */
#define HDARRAY_GEMM_BF16X3 2
#define HDARRAY_GEMM_BF16X6 3
int HDArraySetGemmSplit(int parts);

/* Tile-shape autotuning of the fused stencil launches (also enabled by HDARRAY_AUTOTUNE=1): the
 * first time a stencil plan of a new (kernel, type, partition shape) is compiled in its fused form,
 * the candidate tile shapes are timed on the GPU and the fastest is kept (in memory, and appended
 * to the file named by HDARRAY_TUNE_CACHE if set).  on: 1 or 0. */
int HDArraySetAutotune(int on);

/* Batching: between Begin and End, HDArrayApplyKernel calls do their bookkeeping immediately
 * but their GPU work is deferred; End launches all of it, fused by kernel type into as few
 * launches as possible.  Calls inside one batch must be independent: an array defined by one
 * call may not be used or defined by another call of the batch (HDARRAY_ERR_RACE). */
int HDArrayBatchBegin(void);
int HDArrayBatchEnd(void);

/* CUDA graphs: between Begin and End the library executes normally and records every launch it
 * makes; End captures the recorded launches into a CUDA graph and returns its ID.  Launch
 * replays the graph nrep times; it requires every array the graph touches to be in the exact
 * bookkeeping state it was in at Begin (and, for nrep > 1, the state at End to equal the state
 * at Begin), else HDARRAY_ERR_STATE; after the replays the arrays are in the End state. */
int HDArrayGraphBegin(void);
int HDArrayGraphEnd(int *graphID);
int HDArrayGraphLaunch(int graphID, int nrep);
int HDArrayGraphDestroy(int graphID);

/* Wait for all work of the library stream. */
int HDArraySync(void);

/* Last error recorded by a void call (cleared by reading), and a static message for a code. */
int HDArrayGetLastError(void);
const char *HDArrayErrorString(int code);

/* The exchange of the last call that moved data of hA (ApplyKernel, Read, Reduce): writes up to
 * cap records of 8 int64 each, (src device, dst device, lo0, lo1, lo2, hi0, hi1, hi2) in the
 * user's dimension order (unused dimensions lo 0, hi 1), and returns the number of records
 * (which may exceed cap), or < 0 on error.  The records are disjoint boxes: together they are
 * exactly SENDMSG of Eq. 1 for every (src, dst) pair. */
int64_t HDArrayGetPlan(HDArray_t *hA, int64_t *out, int64_t cap);

/* sGDEF_{p,q} of hA (Sec. 2.1): elements written by device p that device q does not hold, as
 * disjoint boxes, 6 int64 each (lo0, lo1, lo2, hi0, hi1, hi2).  Returns the number of boxes. */
int64_t HDArrayGetGDEF(HDArray_t *hA, int p, int q, int64_t *out, int64_t cap);

/* Device buffer of logical device dev for hA: base pointer, allocated box (user dimension
 * order) and element strides of dimensions 0..2.  *ptr is NULL if the device has no buffer. */
int HDArrayGetDeviceBuffer(HDArray_t *hA, int dev, void **ptr, int64_t *lo, int64_t *hi,
                           int64_t *strides);

/* Copy the raw contents of box [lo, hi) (dim values each, user order) of logical device dev's
 * buffer of hA into the dense host array out (row-major, the box's shape), with no exchange and no
 * bookkeeping: what that device holds, current or stale.  Elements outside the buffer's allocated
 * box are HDARRAY_ERR_RANGE.  For inspection and tests.  Synchronous. */
int HDArrayReadDeviceBuffer(HDArray_t *hA, int dev, const int64_t *lo, const int64_t *hi, void *out);

/* Reduce one strided box of an existing device buffer to one double, allocating nothing.  The paper
 * has no counterpart: HDArrayReduce allocates its scratch and task table with cudaMalloc, which
 * some callers cannot use -- code whose device memory belongs to another allocator (a framework's
 * caching allocator that has reserved the GPU's memory) and latency-critical paths that cannot take
 * cudaMalloc/cudaFree's implicit synchronisation.  This call keeps its scratch (1024 per-CTA
 * partials and a completion counter) in a fixed static device array of the library instead.
 *   x        device pointer to the box's first element; type "double", "float" or "bf16";
 *   extent   dim (1..3) sizes; strides: dim element strides, the innermost must be 1;
 *   op       HDARRAY_SUM / PROD / MAX / MIN, folded in double, deterministic;
 *   result   device pointer to one double that receives the value (caller-owned);
 *   stream   cudaStream_t to run on (NULL: the default stream); the call is asynchronous.
 * The box is spread over up to 1024 CTAs whatever its shape (a 1-D box as well as many short rows).
 * At most 2^31 elements per call (HDARRAY_ERR_RANGE beyond, nothing launched): the limit bounds
 * one call's run time, not the scratch, whose size is fixed; reduce larger boxes in pieces.  The first call on
 * each device looks up the static array's address (with that device current); make it before any
 * stream capture on that device.  Every call shares the static scratch, which keeps the last call's
 * contents (the counter is cleared at the start of each call): calls that overlap on the GPU race
 * and must not be issued concurrently.  Does not touch HDArray bookkeeping. */
int HDArrayReduceBufferNoAlloc(const void *x, const char *type, int dim, const int64_t *extent,
                               const int64_t *strides, REDUCE_OP op, double *result, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* User kernels (extension).  In the paper, users write their own device kernels and give each */
/* array argument use/def clauses, which the frontend turns into the runtime's kernel table     */
/* (Sec. 3, Sec. 4.1).  Here a kernel is a host launcher the runtime calls after the exchange;  */
/* its use/def offsets are set with HDArraySetOffsetUse/Def (or per call with absolute and      */
/* trapezoid sections).                                                                          */
/* ---------------------------------------------------------------------------------------- */

#define HDARRAY_MAX_KERNEL_ARRAYS 8

/* One logical device's share of a call of a user kernel. */
typedef struct {
    int dev;                                          /* logical device */
    int64_t lo[3], hi[3];                             /* work box, in the index space of the
                                                         kernel's space argument (user dimension
                                                         order; unused dimensions lo 0, hi 1) */
    void *buf[HDARRAY_MAX_KERNEL_ARRAYS];             /* device buffer of each array argument on
                                                         this device (NULL if it has none) */
    int64_t buf_lo[HDARRAY_MAX_KERNEL_ARRAYS][3];     /* coordinates of the buffer's first element */
    int64_t buf_stride[HDARRAY_MAX_KERNEL_ARRAYS][3]; /* element strides of dimensions 0..2 */
} HDArrayWork_t;

/* A user kernel's launcher.  HDArrayApplyKernel calls it once per call, after queueing the copies
 * of the incoming sections on the library stream, with the work of every logical device whose
 * work box is not empty (the buffers then hold every element the device uses).  It queues its
 * device work on `stream` (a cudaStream_t), touching only its devices' buffers, and defines exactly
 * the def sections; it returns 0, or a negative code that the apply returns.  It may run during
 * stream capture (HDArrayGraphBegin) and inside batches.  `user` is the pointer given at
 * registration; `work` and `scalars` are valid during the call only. */
typedef int (*HDArrayLauncher_t)(const HDArrayWork_t *work, int nwork, const double *scalars, int nscal,
                                 void *stream, void *user);

/* Register (or replace) the user kernel kName: narr array arguments (at most
 * HDARRAY_MAX_KERNEL_ARRAYS), nscal floating scalars after them, the work partition covering the
 * index space of argument spaceArg.  Every argument's use and def offsets start empty.  A name of a
 * built-in kernel is rejected (HDARRAY_ERR_INVAL). */
int HDArrayRegisterKernel(const char *kName, int narr, int nscal, int spaceArg, HDArrayLauncher_t launcher,
                          void *user);

/* Device memory for array buffers and the library's descriptor tables from a caller-supplied
 * allocator (a framework's caching allocator, say) instead of cudaMalloc / cudaFree.  alloc returns
 * at least `bytes` bytes of device memory aligned to 256 bytes, or NULL; free_fn releases it.
 * (NULL, NULL) restores cudaMalloc / cudaFree.  Takes effect for later allocations: set it before
 * creating arrays; memory is always released by the allocator that provided it, after the device
 * has finished all queued work (as cudaFree would wait). */
typedef void *(*HDArrayAlloc_t)(size_t bytes, void *user);
typedef void (*HDArrayFree_t)(void *ptr, void *user);
int HDArraySetAllocator(HDArrayAlloc_t alloc, HDArrayFree_t free_fn, void *user);

/* ---------------------------------------------------------------------------------------- */
/* Logical devices on several processes (extension).  The paper runs one MPI process per device   */
/* and every process keeps every process's section sets, so all processes compute the same        */
/* messages (Sec. 2.1); messages between processes travel by MPI, messages within one by a device */
/* copy (Sec. 3.1, HDArrayApplyKernel; Sec. 4).  Here each process (a "rank", one GPU each) runs  */
/* the same calls on the same logical devices with the same replicated bookkeeping, holds device  */
/* buffers and runs kernels only for the devices mapped to it, and moves a section whose source   */
/* and destination devices sit on different ranks through a transport the caller supplies.        */
/* ---------------------------------------------------------------------------------------------- */

/* Map logical device d (0 <= d < ndev, ndev = HDArrayNumDevices()) to rank rank_of_dev[d]; this
 * process is rank my_rank.  rank_of_dev NULL (or ndev 0) restores the single-process form, where
 * every device is local.  Set it after HDArrayInit and before creating arrays.  With a map:
 *  - buffers exist, kernels run and Write / Read copy only for this rank's devices;
 *  - HDArrayReduce folds this rank's devices' regions only (combine the ranks' partial results);
 *  - every call whose exchange has a cross-rank section calls the transport (below) after its
 *    bookkeeping and before its kernel, which is then refused inside graph recording
 *    (HDARRAY_ERR_UNSUPPORTED) and without a transport (HDARRAY_ERR_STATE).
 * HDARRAY_ERR_INVAL for a bad map. */
int HDArraySetRankMap(int ndev, const int32_t *rank_of_dev, int my_rank);

/* A cross-rank exchange record: 10 int64, (src device, dst device, src rank, dst rank, lo0, lo1,
 * lo2, hi0, hi1, hi2), the box in the user's dimension order (unused dimensions lo 0, hi 1). */
#define HDARRAY_RANK_RECORD 10

/* The transport: called once per array and call with the nrec cross-rank records of that array's
 * exchange (every rank gets the same records in the same order, sorted by source rank, then
 * destination rank, then the exchange's own order).  It must, before returning, have delivered
 * every record whose dst rank is this rank into its device buffer (HDArrayUnpackBoxes) from the
 * record's src rank, which packs it (HDArrayPackBoxes); the library stream is `stream`.  Returns 0,
 * or a negative code that the call returns. */
typedef int (*HDArrayTransport_t)(HDArray_t *hA, int64_t nrec, const int64_t *recs, void *stream, void *user);
int HDArraySetTransport(HDArrayTransport_t fn, void *user);

/* The cross-rank records (format above, same order as the transport's) of the last call that
 * moved hA's data; up to cap records written, the count returned (which may exceed cap). */
int64_t HDArrayGetRankPlan(HDArray_t *hA, int64_t *out, int64_t cap);

/* Staging layout of nrec records (format above): record i's box in row-major order, element type
 * of hA, starting at the first 16-byte boundary after record i-1.  Returns the total bytes. */
int64_t HDArrayStagingBytes(HDArray_t *hA, int64_t nrec, const int64_t *recs);

/* Pack: copy each record's box from its src device's buffer (a device of this rank) into the
 * staging buffer (device memory, or host memory the GPU can address; layout above, `bytes` at
 * least HDArrayStagingBytes).  Unpack: copy each record's box from staging into its dst device's
 * buffer (a device of this rank), with no bookkeeping (the call that produced the records did it).
 * Queued on the library stream.  HDARRAY_ERR_INVAL if a device is not local, HDARRAY_ERR_RANGE if a
 * box lies outside the device's buffer or staging is too small. */
int HDArrayPackBoxes(HDArray_t *hA, int64_t nrec, const int64_t *recs, void *staging, int64_t bytes);
int HDArrayUnpackBoxes(HDArray_t *hA, int64_t nrec, const int64_t *recs, const void *staging, int64_t bytes);

/* Counters since HDArrayInit: [0] kernel launches issued by the library, [1] section bytes
 * moved between device buffers, [2] plans computed (cache misses), [3] plan cache hits,
 * [4] graph launches.  n values are written (n <= 5). */
int HDArrayGetCounters(int64_t *out, int n);

#ifdef __cplusplus
}
#endif

#endif /* HDARRAY_H */
