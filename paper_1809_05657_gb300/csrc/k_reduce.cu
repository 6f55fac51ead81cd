// k_reduce.cu -- HDArrayReduce (Table 2): fold array sections to one binary64 scalar.
//
// The paper reduces locally on each device and then across processes with MPI (Sec. 3.1, utility
// functions).  Here all logical devices' sections are folded by one launch: CTA b folds tasks
// b, b + G, b + 2G, ... (a warp per row, lanes striding the row), the CTA's warps are combined in
// a fixed shuffle/shared-memory tree, and the last CTA to finish folds the G partials in index
// order.  Nothing depends on scheduling, so the result is reproducible bit for bit.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hda {

template <int DT>
__device__ __forceinline__ double ldd(const void *p, int64_t i);
template <>
__device__ __forceinline__ double ldd<DT_F64>(const void *p, int64_t i)
{
    return reinterpret_cast<const double *>(p)[i];
}
template <>
__device__ __forceinline__ double ldd<DT_F32>(const void *p, int64_t i)
{
    return (double)reinterpret_cast<const float *>(p)[i];
}
template <>
__device__ __forceinline__ double ldd<DT_BF16>(const void *p, int64_t i)
{
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}

template <int OP>
__device__ __forceinline__ double ident()
{
    return OP == 0 ? 0.0 : (OP == 1 ? 1.0 : (OP == 2 ? -__longlong_as_double(0x7ff0000000000000LL)
                                                    : __longlong_as_double(0x7ff0000000000000LL)));
}
template <int OP>
__device__ __forceinline__ double fold(double a, double b)
{
    if (OP == 0) return a + b;
    if (OP == 1) return a * b;
    if (OP == 2) return b > a ? b : a;
    return b < a ? b : a;
}

template <int DT, int OP>
__global__ void __launch_bounds__(256) k_reduce(const RedTask *__restrict__ tasks, int ntasks,
                                                double *partials, unsigned *counter, double *result)
{
    __shared__ double wsum[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // four independent accumulators per lane (column c goes to accumulator (c / 32) % 4), folded
    // together in a fixed order: more loads in flight, same result on every run
    double a0 = ident<OP>(), a1 = a0, a2 = a0, a3 = a0;
    for (int ti = blockIdx.x; ti < ntasks; ti += gridDim.x) {
        const RedTask t = tasks[ti];
        for (int r = t.row_begin + warp; r < t.row_end; r += nw) {
            const int o = r / t.n_mid, m = r - o * t.n_mid;
            const int64_t base = o * t.s_outer + m * t.s_mid;
            int c = lane;
            for (; c + 96 < t.n_inner; c += 128) {
                const double x0 = ldd<DT>(t.x, base + c), x1 = ldd<DT>(t.x, base + c + 32);
                const double x2 = ldd<DT>(t.x, base + c + 64), x3 = ldd<DT>(t.x, base + c + 96);
                a0 = fold<OP>(a0, x0);
                a1 = fold<OP>(a1, x1);
                a2 = fold<OP>(a2, x2);
                a3 = fold<OP>(a3, x3);
            }
            for (int u = 0; c < t.n_inner; c += 32, u++) {
                const double x = ldd<DT>(t.x, base + c);
                if (u == 0) a0 = fold<OP>(a0, x);
                else if (u == 1) a1 = fold<OP>(a1, x);
                else a2 = fold<OP>(a2, x);
            }
        }
    }
    double acc = fold<OP>(fold<OP>(a0, a1), fold<OP>(a2, a3));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = fold<OP>(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = wsum[0];
        for (int w = 1; w < nw; w++) b = fold<OP>(b, wsum[w]);
        partials[blockIdx.x] = b;
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *vp = partials;
        double s = vp[0];
        for (unsigned b = 1; b < gridDim.x; b++) s = fold<OP>(s, vp[b]);
        *result = s;
        *counter = 0u;  // ready for the next launch
    }
}

template <int DT>
static void launch_op(int op, const RedTask *tasks, int ntasks, int nblocks, double *partials,
                      unsigned *counter, double *result, cudaStream_t s)
{
    switch (op) {
    case 0: k_reduce<DT, 0><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result); break;
    case 1: k_reduce<DT, 1><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result); break;
    case 2: k_reduce<DT, 2><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result); break;
    default: k_reduce<DT, 3><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result); break;
    }
}

cudaError_t launch_reduce(int dtype, int op, const RedTask *tasks, int ntasks, int nblocks,
                          double *partials, unsigned *counter, double *result, cudaStream_t s)
{
    if (nblocks < 1 || op < 0 || op > 3) return cudaErrorInvalidValue;
    switch (dtype) {
    case DT_F64: launch_op<DT_F64>(op, tasks, ntasks, nblocks, partials, counter, result, s); break;
    case DT_F32: launch_op<DT_F32>(op, tasks, ntasks, nblocks, partials, counter, result, s); break;
    case DT_BF16: launch_op<DT_BF16>(op, tasks, ntasks, nblocks, partials, counter, result, s); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hda
