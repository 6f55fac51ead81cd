// kernels.h -- device-side descriptors and host launchers of the library's CUDA kernels.
//
// All tables are built by the host runtime once per plan (a cached exchange + kernel for one
// HDArrayApplyKernel signature and GDEF state), uploaded to device memory, and then reused by
// every launch that replays the plan.  Pointers inside the tables are device addresses.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hda {

enum DType { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2 };

// ------------------------------------------------------------------------------------------
// Section copy: the exchange of Eq. 1-2 moved between two device buffers.  A box is viewed as
// n_outer x n_mid rows of `inner` contiguous bytes.  One task is a slice of rows of one box.
// ------------------------------------------------------------------------------------------
struct CopyTask {
    const char *src;  // first byte of the box in the source buffer
    char *dst;        // first byte of the box in the destination buffer
    int64_t s_outer, s_mid;  // source byte strides
    int64_t d_outer, d_mid;  // destination byte strides
    int32_t n_mid;           // rows per outer index
    int32_t inner;           // contiguous bytes per row
    int32_t row_begin, row_end;  // rows [row_begin, row_end) of the flattened outer*mid range
    int32_t vec;             // widest access (16, 8, 4 or 2 bytes) all addresses and `inner` allow
    int32_t pad;
};
cudaError_t launch_copy(const CopyTask *tasks, int ntasks, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// 2-D 4-neighbour Jacobi step (Sec. 5), fused with the exchange.
// A tile is one warp's job: output rows [r0, r1) x columns [c0, c1) inside one column band of
// 32 vector chunks starting at cb.  Before computing, the warp copies its receive segments (the
// parts of the device's incoming sections that only this tile reads) from the sender's buffer
// into its own buffer.
// ------------------------------------------------------------------------------------------
struct StenPart2D {
    const void *x;  // X buffer (used array) of this device
    void *y;        // Y buffer (defined array) of this device
    int64_t xlo0, xlo1, xs;  // X buffer origin (row, col) and row stride in elements
    int64_t ylo0, ylo1, ys;
    int32_t rwb;  // TMA variant: width of the part's staged rows in 16-byte chunks (band + 2 halo chunks)
    int32_t pad_;
};
struct StenTile2D {
    int32_t part;
    int32_t r0, r1;
    int32_t c0, c1;
    int32_t cb;
    int32_t seg0, nseg;
    int32_t nch, ns, sl;  // packed-stream variant: chunks per row, streams, rows per stream;
                          // TMA variant: chunks per row, row groups of JACOBI2D_TMA_ROWS rows
};
struct Seg {  // dst[o * dso + k * ds] = src[o * sso + k * ss], k < n, o < m (element strides)
    const void *src;
    void *dst;
    int64_t ss, ds;    // inner strides
    int64_t sso, dso;  // outer strides
    int32_t n, m;
};
// variant 0: a warp per tile, prefetched rows in registers; variant 1: a warp per tile, rows in
// shared memory via cp.async (warps_per_cta tiles per CTA); variant 3: a CTA per tile of ns row
// streams x nch chunks, rows in a shared-memory ring of JACOBI2D_STAGES stages of smem / (16 *
// JACOBI2D_STAGES) >= ns * (nch + 2) slots (at most 512).
constexpr int JACOBI2D_STAGES = 8;
cudaError_t launch_jacobi2d(int dtype, const StenPart2D *parts, const StenTile2D *tiles,
                            int ntiles, const Seg *segs, int warps_per_cta, int variant, size_t smem,
                            cudaStream_t s);
// variant 5: a CTA of 256 threads per tile of nch chunks x rows r0 .. r1 - 1, cut into stages of
// ns * JACOBI2D_TMA_ROWS output rows (ns * nch <= 256), each stage one bulk tensor copy of its rows
// and the two halo rows by the part's rwb chunks into a ring of JACOBI2D_TMA_STAGES stages (each
// padded to 128 bytes; smem = the ring + 128 bytes of alignment slack, at most
// JACOBI2D_TMA_SMEM_MAX).  tmaps holds one 128-byte CUtensorMap per part (its X buffer, box
// rwb * 16 bytes x (ns * rows + 2)); err receives a set bit when a bounded wait gave up after
// spin_limit polls.  rx_cap > 0 (a multiple of 256, at most JACOBI2D_TMA_RX_MAX): a tile with at
// most rx_cap received elements issues its first copies before its receive and patches the
// received values into those stages; the launch adds rx_cap * (element size + 4) bytes of shared
// memory after the ring for them.  Tiles with more, and every tile when rx_cap = 0, receive first.
constexpr int JACOBI2D_TMA_STAGES = 4;
constexpr int JACOBI2D_TMA_ROWS = 4;
constexpr int JACOBI2D_TMA_THREADS = 256;
constexpr int JACOBI2D_TMA_STAGE_MAX = 20 * 1024;  // largest stage the tile planner makes
constexpr int JACOBI2D_TMA_RX_MAX = 4 * JACOBI2D_TMA_THREADS;
constexpr int JACOBI2D_TMA_SMEM_MAX =
    JACOBI2D_TMA_STAGES * (JACOBI2D_TMA_STAGE_MAX + 128) + 128 + JACOBI2D_TMA_RX_MAX * (8 + 4);
// op 0: the Jacobi step; op 1: the 3 x 3 convolution of launch_stencil2d_cta with weights[9].
cudaError_t launch_jacobi2d_tma(int op, int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                const Seg *segs, size_t smem, cudaStream_t s, const void *tmaps, const double *weights,
                                unsigned *err, unsigned spin_limit, int rx_cap);
// The packed-stream kernel with a chosen point operation: op 0 the Jacobi step, op 1 the 3 x 3
// convolution with weights[9] (device memory, binary64, row-major over the offsets
// (-1,-1) (-1,0) (-1,1) (0,-1) ... (1,1)).
cudaError_t launch_stencil2d_cta(int op, int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                 const Seg *segs, const double *weights, size_t smem, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// 3-D 7-point step, fused with the exchange.  Per-warp variant: a tile is one warp's job, output
// row y, x in [x0, x1) inside a band of 32 vector chunks starting at xb, marching z over [z0, z1);
// consecutive tiles are consecutive rows, so the rows y-1 and y+1 a warp reads were just read by
// its neighbours in the same CTA.  CTA variant: a tile is ny rows x nch chunks from xb (one chunk
// per thread of a 256- or 512-thread CTA), x in [x0, x1), marching z over [z0, z1).
// ------------------------------------------------------------------------------------------
struct StenPart3D {
    const void *x;
    void *y;
    int64_t xlo0, xlo1, xlo2, xs0, xs1;  // origin (z, y, x) and strides of z and y (elements)
    int64_t ylo0, ylo1, ylo2, ys0, ys1;
    int32_t rwb, boxh;  // TMA variant: staged plane box of the part's tiles, 16-byte chunks x rows
};
struct StenTile3D {
    int32_t part;
    int32_t z0, z1;
    int32_t y;   // first row
    int32_t x0, x1;
    int32_t xb;
    int32_t seg0, nseg;
    int32_t ny;   // rows: 1 for the per-warp variant, ny * nch <= threads for the CTA variant
    int32_t nch;  // 16-byte chunks per row from xb (CTA variant; (ny + 2) * (nch + 2) <= 2 * threads)
};
// Plane-ring depth of the CTA variant; its dynamic shared memory is
// STENCIL3D_STAGES * max over tiles of (ny + 2) * (nch + 2) * 16 bytes.
constexpr int STENCIL3D_STAGES = 8;
// variant 0: one warp per tile (a row), prefetch in registers (warps_per_cta tiles per CTA);
// variant 1: one CTA of 32 * warps_per_cta threads (8 or 16 warps) per tile, planes prefetched into
// shared memory (cp.async), smem bytes as above.
// variant 3 (the CTA tiles with planes staged by TMA): tmaps holds one 128-byte CUtensorMap per
// part (its X buffer), err receives a set bit when a bounded wait gave up after spin_limit polls.
cudaError_t launch_stencil3d(int dtype, const StenPart3D *parts, const StenTile3D *tiles,
                             int ntiles, const Seg *segs, int warps_per_cta, int variant, size_t smem,
                             cudaStream_t s, const void *tmaps = nullptr, unsigned *err = nullptr,
                             unsigned spin_limit = 0);

// Flat-block forms (binary32 / binary64): one CTA per block of a work box, the block and its halo
// staged in shared memory, threads walking the block's cells in row-major order.  2-D tiles use
// r0, r1, c0, c1 (cb unused); 3-D tiles use z0, z1, y, ny, x0, x1 (xb unused).
constexpr int FLAT3D_STAGES = 6;
size_t flat2d_smem(int dtype, int rows, int cols);
size_t flat3d_smem(int dtype, int ny, int nx);
cudaError_t launch_jacobi2d_flat(int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                 const Seg *segs, size_t smem, cudaStream_t s);
cudaError_t launch_stencil3d_flat(int dtype, const StenPart3D *parts, const StenTile3D *tiles, int ntiles,
                                  const Seg *segs, size_t smem, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Element-wise residual R = (X - Y)^2 in double over boxes.
// ------------------------------------------------------------------------------------------
struct PwTask {
    const void *x;
    const void *y;
    double *r;
    int64_t xs_outer, xs_mid, ys_outer, ys_mid, rs_outer, rs_mid;  // element strides
    int32_t n_mid, n_inner;
    int32_t row_begin, row_end;
};
// With partials == nullptr: one CTA per task, R only.  Otherwise `nblocks` CTAs also fold the sum of
// the stored values: partials (nblocks doubles), counter (zero on entry, left zero), result.
cudaError_t launch_sqdiff(int dtype, const PwTask *tasks, int ntasks, int nblocks, double *partials,
                          unsigned *counter, double *result, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Reduction of boxes to one double (HDArrayReduce, Table 2).  Deterministic: the task list and
// the grid are fixed, every CTA folds a fixed set of rows in a fixed order, and the last CTA to
// finish folds the per-CTA partials in index order.
// ------------------------------------------------------------------------------------------
struct RedTask {
    const void *x;
    int64_t s_outer, s_mid;  // element strides
    int32_t n_mid, n_inner;
    int32_t row_begin, row_end;
};
// scratch: `nblocks` doubles of partials followed by one unsigned counter (zero on entry, left
// zero on exit); result: one double.
cudaError_t launch_reduce(int dtype, int op, const RedTask *tasks, int ntasks, int nblocks,
                          double *partials, unsigned *counter, double *result, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// GEMM of Listing 3 over row blocks: C[i][j] = beta*C[i][j] + alpha * sum_k A[i][k] * B[k][j],
// for work rows [i0, i1) and all columns, A lower triangular when `lower` (k <= i only).
// ------------------------------------------------------------------------------------------
struct GemmPart {
    const void *a;
    const void *b;
    void *c;
    int64_t alo0, alo1, as;  // buffer origins (row, col) and row strides (elements)
    int64_t blo0, blo1, bs;
    int64_t clo0, clo1, cs;
    int32_t i0, i1, j0, j1;  // work box of C
    int32_t nk;
    int32_t lower;   // A lower triangular (k <= i only)
    int32_t transa;  // A[i][k] is element (k, i) of the A buffer (C = alpha X^T X: syrk)
    int32_t upper;   // only the elements with j >= i of C are computed and stored
};
cudaError_t launch_gemm_f64(const GemmPart *parts, int nparts, int max_rows, int max_cols,
                            double alpha, double beta, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// The same GEMM on binary32 arrays with the tensor cores (bf16x3 split, binary32 accumulation).
// One CTA per 128 x 256 tile of C; kend = the K extent the tile needs (triangular A: its last row
// + 1).  *err is set if a bounded wait gave up.
// ------------------------------------------------------------------------------------------
struct TcPart {
    const void *a;
    const void *b;
    void *c;
    int64_t alo0, alo1, as;
    int64_t blo0, blo1, bs;
    int64_t clo0, clo1, cs;
    int32_t i1, j1;  // ends of the device's work box (rows, columns)
    int32_t lower;
    int32_t pad;
};
struct TcTile {
    int32_t part;
    int32_t i0, j0;
    int32_t kend;
};
size_t gemm_tc_smem_bytes();

// Pre-split bf16 hi/lo operand panels (see k_gemm_tc.cu for the layout) and the pipelined GEMM
// that streams them with bulk copies.
struct SplitJob {
    const void *src;   // binary32 buffer
    void *dst;         // panel
    int64_t lo0, lo1, stride;  // buffer origin (row, col) and row stride (elements)
    int32_t row0, row_end;     // A: rows of C's row tiles; B: columns of C's column tiles
    int32_t kend;              // K extent
    int32_t nkt, ntiles;       // k tiles per row tile, total tiles
    int32_t rows_per_tile;     // 128 (A) or the GEMM's CTA width (B: 256)
    int32_t transpose;         // 1 for B (stored as B^T)
    int32_t lower;             // A lower triangular
    int32_t nparts;            // bf16 parts per value: 2 (hi, lo) or 3 (hi, mid, lo)
    int32_t bk;                // k per tile: 64 (128-byte rows, 2 parts) or 32 (64-byte rows, 3 parts)
};
struct PanelPart {
    const void *apanel;  // A panel of this device's rows (row tiles from row0)
    const void *bpanel;  // B panel of this device's columns (column tiles from col0)
    void *c;
    int64_t clo0, clo1, cs;
    int32_t row0;        // first row of the device's row tiles
    int32_t i1, j1;
    int32_t nkt, nkt_b;  // k tiles per row tile in the A and B panels
    int32_t col0;        // first column of the device's column tiles
    int32_t upper;       // store only the elements with j >= i
    int32_t nparts;      // bf16 parts per operand value: 2 (bf16x3) or 3 (bf16x6)
};
cudaError_t launch_split_panels(const SplitJob *jobs, int njobs, int max_tiles, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// Covariance pieces (Sec. 5.1).  A task is one logical device's work box.
// colmean: M[0][j] = (sum over the n rows of X[i][j]) / n for j in [j0, j1), binary64 sums in a
//          fixed order (deterministic), or (mode 1) sqrt(sum of X[i][j]^2);
// centre: Xc = X - M, or (mode 1) X / M, over [i0, i1) x [j0, j1);
// symmetrize: C[i][j] = C[j][i] for the elements with j < i of [i0, i1) x [j0, j1).
// ------------------------------------------------------------------------------------------
struct CovTask {
    const void *x;  // colmean, centre: X; symmetrize: C (read at the transposed positions)
    const void *m;  // colmean: M (written); centre: M (read)
    void *y;        // centre: Xc; symmetrize: C (written)
    int64_t xlo0, xlo1, xs;
    int64_t mlo1;   // M's buffer origin column (its one row is row 0)
    int64_t ylo0, ylo1, ys;
    int32_t i0, i1, j0, j1;
    int32_t n;      // colmean: the rows of X
    int32_t mode;   // colmean: 0 mean, 1 root of the sum of squares; centre: 0 X - M, 1 X / M
};
cudaError_t launch_colmean(int dtype, const CovTask *tasks, int ntasks, int max_cols, cudaStream_t s);
cudaError_t launch_center(int dtype, const CovTask *tasks, int ntasks, int max_rows, cudaStream_t s);
cudaError_t launch_symmetrize(int dtype, const CovTask *tasks, int ntasks, int max_rows, int max_cols,
                              cudaStream_t s);
// spin_limit: polls of each pipeline wait before the kernel gives up (sets *err); the waits for
// copies and MMAs already issued always use the fixed limit.
constexpr unsigned GEMM_SPIN_LIMIT_DEFAULT = 1u << 24;
// nparts 2: bf16x3 products, 128 x 256 CTA tiles; 3: bf16x6 products, 128 x 128 CTA tiles.
cudaError_t launch_gemm_panels(const PanelPart *parts, const TcTile *tiles, int ntiles, float alpha,
                               float beta, unsigned *err, unsigned spin_limit, int nparts, cudaStream_t s);
cudaError_t launch_gemm_tc(const TcPart *parts, const TcTile *tiles, int ntiles, float alpha, float beta,
                           unsigned *err, cudaStream_t s);

}  // namespace hda
