// k_gemm.cu -- the GEMM kernel of Listing 3 in binary64 on every logical device's row block:
//
//   C[i][j] = beta * C[i][j] + alpha * sum_k A[i][k] * B[k][j]
//
// with A optionally lower triangular (k <= i only; the elements above the diagonal are outside
// the device's use section and are never read).  Each device reads its own A rows and C rows and
// the whole of B, which the exchange has gathered into its buffer (Sec. 5.1: GEMM all-gathers B).
//
// A plain shared-memory tiled DFMA kernel: 64 x 64 C tile per CTA, 256 threads with 4 x 4
// outputs each, K in steps of 16.  This is the binary64 comparison form.  It also serves the
// covariance product C = alpha X^T X (A read transposed, only j >= i computed).
#include "kernels.h"

namespace hda {

constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_gemm_f64(const GemmPart *__restrict__ parts,
                                                  double alpha, double beta)
{
    const GemmPart P = parts[blockIdx.z];
    const int i0 = P.i0 + blockIdx.y * GT, j0 = P.j0 + blockIdx.x * GT;
    if (i0 >= P.i1 || j0 >= P.j1) return;
    if (P.upper && j0 + GT - 1 < i0) return;  // the tile lies below the diagonal
    const int ie = min(i0 + GT, P.i1);
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT];
    const double *A = reinterpret_cast<const double *>(P.a);
    const double *B = reinterpret_cast<const double *>(P.b);
    double *C = reinterpret_cast<double *>(P.c);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    const int kend = P.lower ? min(P.nk, ie) : P.nk;
    for (int k0 = 0; k0 < kend; k0 += GK) {
        // A tile: 64 rows x 16 k, transposed into As[k][i] (consecutive threads on consecutive
        // addresses: along k for a row-major A, along i for a transposed one)
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int ii = P.transa ? e % GT : e / GK, kk = P.transa ? e / GT : e % GK;
            const int i = i0 + ii, k = k0 + kk;
            double v = 0.0;
            if (i < P.i1 && k < kend && (!P.lower || k <= i))
                v = P.transa ? A[(int64_t)(k - P.alo0) * P.as + (i - P.alo1)]
                             : A[(int64_t)(i - P.alo0) * P.as + (k - P.alo1)];
            As[kk][ii] = v;
        }
        // B tile: 16 k x 64 columns
        for (int e = threadIdx.x; e < GT * GK; e += 256) {
            const int kk = e / GT, jj = e % GT;
            const int k = k0 + kk, j = j0 + jj;
            double v = 0.0;
            if (k < kend && j < P.j1) v = B[(int64_t)(k - P.blo0) * P.bs + (j - P.blo1)];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) a[u] = As[kk][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; v++) b[v] = Bs[kk][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int i = i0 + ty * 4 + u;
        if (i >= P.i1) continue;
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int j = j0 + tx * 4 + v;
            if (j >= P.j1 || (P.upper && j < i)) continue;
            double *c = C + (int64_t)(i - P.clo0) * P.cs + (j - P.clo1);
            const double old = beta == 0.0 ? 0.0 : *c;
            *c = beta * old + alpha * acc[u][v];
        }
    }
}

cudaError_t launch_gemm_f64(const GemmPart *parts, int nparts, int max_rows, int max_cols,
                            double alpha, double beta, cudaStream_t s)
{
    if (nparts <= 0 || max_rows <= 0 || max_cols <= 0) return cudaSuccess;
    dim3 grid((max_cols + GT - 1) / GT, (max_rows + GT - 1) / GT, nparts);
    k_gemm_f64<<<grid, 256, 0, s>>>(parts, alpha, beta);
    return cudaGetLastError();
}

}  // namespace hda
