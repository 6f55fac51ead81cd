// k_cov.cu -- the element-wise and copy pieces of the covariance and correlation programs
// (Sec. 5.1): column means and norms, centring and scaling, and the symmetric copy that completes
// the triangular product.  The product
// itself (C = alpha X^T X, j >= i) runs on the GEMM kernels (k_gemm.cu, k_gemm_tc.cu).
#include "kernels.h"

namespace hda {

template <typename T>
__device__ __forceinline__ double ld64(const T *p) { return (double)*p; }

// Column means (or norms): one CTA per (device, 32 columns); lane = column, warp w sums the rows
// w, w+8, ... (or their squares) in binary64, then the eight partial sums are folded in warp order
// (a fixed order: the result does not depend on scheduling).
template <typename T>
__global__ void __launch_bounds__(256) k_colmean(const CovTask *__restrict__ tasks)
{
    const CovTask t = tasks[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = t.j0 + blockIdx.x * 32 + lane;
    __shared__ double part[8][32];
    double s = 0.0;
    if (t.j0 + blockIdx.x * 32 < t.j1 && j < t.j1) {
        const T *x = reinterpret_cast<const T *>(t.x) + (j - t.xlo1);
        if (t.mode == 0) {
            for (int i = warp; i < t.n; i += 8) s += ld64(x + (int64_t)(i - t.xlo0) * t.xs);
        } else {
            for (int i = warp; i < t.n; i += 8) {
                const double v = ld64(x + (int64_t)(i - t.xlo0) * t.xs);
                s += v * v;
            }
        }
    }
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && t.j0 + blockIdx.x * 32 < t.j1 && j < t.j1) {
        double a = part[0][lane];
#pragma unroll
        for (int w = 1; w < 8; w++) a += part[w][lane];
        T *m = const_cast<T *>(reinterpret_cast<const T *>(t.m));
        m[j - t.mlo1] = (T)(t.mode == 0 ? a / (double)t.n : sqrt(a));
    }
}

// Centring (or scaling): a warp per row of the device's box, four loads in flight per lane; one
// IEEE subtraction (or division) per element in the storage precision.
template <typename T>
__global__ void __launch_bounds__(256) k_center(const CovTask *__restrict__ tasks)
{
    const CovTask t = tasks[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = t.i0 + blockIdx.x * 8 + warp;
    if (i >= t.i1) return;
    const T *x = reinterpret_cast<const T *>(t.x) + (int64_t)(i - t.xlo0) * t.xs - t.xlo1;
    const T *m = reinterpret_cast<const T *>(t.m) - t.mlo1;
    T *y = reinterpret_cast<T *>(t.y) + (int64_t)(i - t.ylo0) * t.ys - t.ylo1;
    for (int j = t.j0 + lane; j < t.j1; j += 128) {
        T a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (j + 32 * u < t.j1) {
                a[u] = x[j + 32 * u];
                b[u] = m[j + 32 * u];
            }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (j + 32 * u < t.j1) y[j + 32 * u] = t.mode == 0 ? a[u] - b[u] : a[u] / b[u];
    }
}

// Symmetric copy: 32 x 32 tiles of the device's box on or below the diagonal; the transposed
// tile C[j][i] is read row-wise into shared memory and written as C[i][j] for j < i.
template <typename T>
__global__ void __launch_bounds__(256) k_symmetrize(const CovTask *__restrict__ tasks)
{
    const CovTask t = tasks[blockIdx.z];
    const int ti = t.i0 + blockIdx.y * 32, tj = t.j0 + blockIdx.x * 32;
    if (ti >= t.i1 || tj >= t.j1 || tj > ti + 31) return;  // outside the box or above the diagonal
    __shared__ T tile[32][33];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const T *c = reinterpret_cast<const T *>(t.x);
    for (int r = ly; r < 32; r += 8) {  // rows j = tj + r of the transposed tile, columns i = ti + lx
        const int j = tj + r, i = ti + lx;
        if (j < t.j1 && i < t.i1 && j < i) tile[r][lx] = c[(int64_t)(j - t.xlo0) * t.xs + (i - t.xlo1)];
    }
    __syncthreads();
    T *y = reinterpret_cast<T *>(t.y);
    for (int r = ly; r < 32; r += 8) {  // rows i = ti + r, columns j = tj + lx
        const int i = ti + r, j = tj + lx;
        if (i < t.i1 && j < t.j1 && j < i) y[(int64_t)(i - t.ylo0) * t.ys + (j - t.ylo1)] = tile[lx][r];
    }
}

cudaError_t launch_colmean(int dtype, const CovTask *tasks, int ntasks, int max_cols, cudaStream_t s)
{
    if (ntasks <= 0 || max_cols <= 0) return cudaSuccess;
    dim3 grid((max_cols + 31) / 32, ntasks);
    if (dtype == DT_F64) k_colmean<double><<<grid, 256, 0, s>>>(tasks);
    else if (dtype == DT_F32) k_colmean<float><<<grid, 256, 0, s>>>(tasks);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_center(int dtype, const CovTask *tasks, int ntasks, int max_rows, cudaStream_t s)
{
    if (ntasks <= 0 || max_rows <= 0) return cudaSuccess;
    dim3 grid((max_rows + 7) / 8, ntasks);
    if (dtype == DT_F64) k_center<double><<<grid, 256, 0, s>>>(tasks);
    else if (dtype == DT_F32) k_center<float><<<grid, 256, 0, s>>>(tasks);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_symmetrize(int dtype, const CovTask *tasks, int ntasks, int max_rows, int max_cols,
                              cudaStream_t s)
{
    if (ntasks <= 0 || max_rows <= 0 || max_cols <= 0) return cudaSuccess;
    dim3 grid((max_cols + 31) / 32, (max_rows + 31) / 32, ntasks);
    if (dtype == DT_F64) k_symmetrize<double><<<grid, 256, 0, s>>>(tasks);
    else if (dtype == DT_F32) k_symmetrize<float><<<grid, 256, 0, s>>>(tasks);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace hda
