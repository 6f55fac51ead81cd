// k_reduce.cu -- HDArrayReduce (Table 2): fold array sections to one binary64 scalar.
//
// The paper reduces locally on each device and then across processes with MPI (Sec. 3.1, utility
// functions).  Here all logical devices' sections are folded by one launch: CTA b folds tasks
// b, b + G, b + 2G, ... (a warp per row, lanes striding the row), the CTA's warps are combined in
// a fixed shuffle/shared-memory tree, and the last CTA to finish folds the G partials in index
// order.  Nothing depends on scheduling, so the result is reproducible bit for bit.
#include <cuda_bf16.h>

#include "exact_sqdiff.h"
#include "kernels.h"

namespace hda {

// binary32 -> binary64 by integer operations (exact, like the conversion instruction, which on
// this GPU runs in the slow binary64 pipe): a normal number keeps its sign and significand and
// moves its exponent bias from 127 to 1023; a subnormal is normalised; infinities and NaNs keep
// their payload (NaNs made quiet).
__device__ __forceinline__ double f32_bits_to_f64(unsigned u)
{
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e - 1u < 254u)  // normal: exponent field e + (1023 - 127)
        return __longlong_as_double((long long)(sign | (((unsigned long long)(u & 0x7fffffffu) << 29) +
                                                        (896ull << 52))));
    unsigned long long bits;
    if (e == 0xffu) {
        bits = sign | 0x7ff0000000000000ull | ((unsigned long long)m << 29);
        if (m) bits |= 0x0008000000000000ull;
    } else if (m == 0) {
        bits = sign;
    } else {  // m * 2^-149 with the top bit of m at position k: exponent field k - 149 + 1023
        const int k = 31 - __clz(m);
        bits = sign | ((unsigned long long)(k + 874) << 52) |
               (((unsigned long long)m << (52 - k)) & 0x000fffffffffffffull);
    }
    return __longlong_as_double((long long)bits);
}

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
    return f32_bits_to_f64(reinterpret_cast<const unsigned *>(p)[i]);
}
template <>
__device__ __forceinline__ double ldd<DT_BF16>(const void *p, int64_t i)
{
    return f32_bits_to_f64((unsigned)reinterpret_cast<const unsigned short *>(p)[i] << 16);
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

// ------------------------------------------------------------------------------------------
// R = (X - Y)^2 in binary64 over boxes (the residual field of the Jacobi program), optionally
// folding the stored values' sum on the way (SUM partials per CTA, the last CTA folds them into
// `result`): HDArrayReduce(R, SUM) over the same boxes then needs no second pass over R.
//
// Work: CTA b takes tasks b, b + G, ...; a warp per row.  Every buffer's rows share one 16-byte
// phase (element c is 16-byte aligned in x, y and r alike once the head is done), so a row is a
// scalar head up to x's first 16-byte boundary, then 16-byte vectors of x and y (V elements)
// with V doubles of r stored per vector, two vectors in flight per lane, then a scalar tail.  A
// row whose y or r does not share x's phase runs scalar.  Each lane folds its elements in a
// fixed order and the trees are fixed, so the sum is the same on every run of a plan.
// ------------------------------------------------------------------------------------------
// 16 bytes of a stored row: V elements, as binary64 values (binary64 storage) or as binary32 bit
// patterns (binary32 and bfloat16 storage; bfloat16 -> binary32 is exact: the bits move up 16
// places).
template <int DT>
struct Vec16;
template <>
struct Vec16<DT_F64> {
    static constexpr int V = 2;
    using T = double;
    __device__ static void load(const void *p, double *out)
    {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        out[0] = v.x;
        out[1] = v.y;
    }
    __device__ static double one(const void *p, int c) { return reinterpret_cast<const double *>(p)[c]; }
};
template <>
struct Vec16<DT_F32> {
    static constexpr int V = 4;
    using T = unsigned;
    __device__ static void load(const void *p, unsigned *out)
    {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    }
    __device__ static unsigned one(const void *p, int c) { return reinterpret_cast<const unsigned *>(p)[c]; }
};
template <>
struct Vec16<DT_BF16> {
    static constexpr int V = 8;
    using T = unsigned;
    __device__ static void load(const void *p, unsigned *out)
    {
        const uint4 v = *reinterpret_cast<const uint4 *>(p);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            out[2 * k] = w[k] << 16;
            out[2 * k + 1] = w[k] & 0xffff0000u;
        }
    }
    __device__ static unsigned one(const void *p, int c)
    {
        return (unsigned)reinterpret_cast<const unsigned short *>(p)[c] << 16;
    }
};

// RN64((x - y)^2) of two stored elements
__device__ __forceinline__ double sq_of(double a, double b)
{
    const double d = a - b;
    return d * d;
}
__device__ __forceinline__ double sq_of(unsigned ux, unsigned uy)
{
    uint64_t q;
    if (sqdiff_f32_exact(__uint_as_float(ux), __uint_as_float(uy), q))           // exact difference
        return __longlong_as_double((long long)q);
    if (sqdiff_f32_bits(ux, uy, q)) return __longlong_as_double((long long)q);  // integer path
    const double d = f32_bits_to_f64(ux) - f32_bits_to_f64(uy);                 // the rest
    return d * d;
}

template <int DT, bool SUM>
__global__ void __launch_bounds__(256) k_sqdiff(const PwTask *__restrict__ tasks, int ntasks, double *partials,
                                                unsigned *counter, double *result)
{
    using VT = Vec16<DT>;
    using T = typename VT::T;
    constexpr int V = VT::V;
    constexpr int ES = 16 / V;  // bytes per stored element of x and y
    __shared__ double wsum[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double acc = 0.0;
    for (int ti = blockIdx.x; ti < ntasks; ti += gridDim.x) {
        const PwTask t = tasks[ti];
        const int n = t.n_inner;
        for (int row = t.row_begin + warp; row < t.row_end; row += nw) {
            const int o = row / t.n_mid, m = row - o * t.n_mid;
            const char *x = reinterpret_cast<const char *>(t.x) + (o * t.xs_outer + m * t.xs_mid) * ES;
            const char *y = reinterpret_cast<const char *>(t.y) + (o * t.ys_outer + m * t.ys_mid) * ES;
            double *r = t.r + o * t.rs_outer + m * t.rs_mid;
            int head = (int)(((16 - ((uintptr_t)x & 15)) & 15) / ES);
            if (head > n) head = n;
            const bool vec = (((uintptr_t)(y + head * ES) | (uintptr_t)(r + head)) & 15) == 0;
            const int nv = vec ? (n - head) / V : 0;
            const int vend = vec ? head + nv * V : 0;
            auto scalar = [&](int c) {
                const double q = sq_of(VT::one(x, c), VT::one(y, c));
                r[c] = q;
                if (SUM) acc += q;
            };
            // scalar head (head < V <= 8 elements), then the tail after the vectors; a row
            // without a common phase is all tail (vend = 0)
            if (vec && lane < head) scalar(lane);
            for (int c = vend + lane; c < n; c += 32) scalar(c);
            int v = lane;
            for (; v + 32 < nv; v += 64) {  // two vectors in flight per lane
                T a0[V], b0[V], a1[V], b1[V];
                VT::load(x + (head + v * V) * ES, a0);
                VT::load(y + (head + v * V) * ES, b0);
                VT::load(x + (head + (v + 32) * V) * ES, a1);
                VT::load(y + (head + (v + 32) * V) * ES, b1);
                double q0[V], q1[V];
#pragma unroll
                for (int k = 0; k < V; k++) {
                    q0[k] = sq_of(a0[k], b0[k]);
                    q1[k] = sq_of(a1[k], b1[k]);
                }
                double2 *r0 = reinterpret_cast<double2 *>(r + head + v * V);
                double2 *r1 = reinterpret_cast<double2 *>(r + head + (v + 32) * V);
#pragma unroll
                for (int k = 0; k < V / 2; k++) {
                    r0[k] = make_double2(q0[2 * k], q0[2 * k + 1]);
                    r1[k] = make_double2(q1[2 * k], q1[2 * k + 1]);
                }
                if (SUM) {
#pragma unroll
                    for (int k = 0; k < V; k++) acc += q0[k];
#pragma unroll
                    for (int k = 0; k < V; k++) acc += q1[k];
                }
            }
            for (; v < nv; v += 32) {
                T a0[V], b0[V];
                double q0[V];
                VT::load(x + (head + v * V) * ES, a0);
                VT::load(y + (head + v * V) * ES, b0);
#pragma unroll
                for (int k = 0; k < V; k++) q0[k] = sq_of(a0[k], b0[k]);
                double2 *r0 = reinterpret_cast<double2 *>(r + head + v * V);
#pragma unroll
                for (int k = 0; k < V / 2; k++) r0[k] = make_double2(q0[2 * k], q0[2 * k + 1]);
                if (SUM) {
#pragma unroll
                    for (int k = 0; k < V; k++) acc += q0[k];
                }
            }
        }
    }
    if (SUM) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) wsum[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = wsum[0];
            for (int w = 1; w < nw; w++) b += wsum[w];
            partials[blockIdx.x] = b;
            __threadfence();
            last = (atomicAdd(counter, 1u) == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            const volatile double *vp = partials;
            double s = vp[0];
            for (unsigned b = 1; b < gridDim.x; b++) s += vp[b];
            *result = s;
            *counter = 0u;  // ready for the next launch
        }
    }
}

cudaError_t launch_sqdiff(int dtype, const PwTask *tasks, int ntasks, int nblocks, double *partials,
                          unsigned *counter, double *result, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    const bool sum = partials != nullptr;
    if (!sum || nblocks < 1) nblocks = ntasks;
    switch (dtype) {
    case DT_F64:
        if (sum) k_sqdiff<DT_F64, true><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        else k_sqdiff<DT_F64, false><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        break;
    case DT_F32:
        if (sum) k_sqdiff<DT_F32, true><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        else k_sqdiff<DT_F32, false><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        break;
    case DT_BF16:
        if (sum) k_sqdiff<DT_BF16, true><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        else k_sqdiff<DT_BF16, false><<<nblocks, 256, 0, s>>>(tasks, ntasks, partials, counter, result);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
