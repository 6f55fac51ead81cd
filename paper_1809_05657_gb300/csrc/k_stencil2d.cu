// k_stencil2d.cu -- the Jacobi step of Sec. 5 on every logical device's work region, fused with
// the exchange, plus the element-wise residual kernel.
//
//   Y[i][j] = (X[i][j-1] + X[i][j+1] + X[i-1][j] + X[i+1][j]) / 4
//
// summed left to right as printed, in the storage precision (binary64 or binary32) or, for
// bfloat16 storage, in binary32 with one round-to-nearest-even on the store.  The division by 4 is
// a multiplication by 0.25, which is exact scaling and so gives the same bits.
//
// Work decomposition: one warp per tile.  A tile is a column band of 32 lanes x one 16-byte
// chunk per lane (4 floats, 2 doubles or 8 bfloat16) and a run of rows; the warp marches down the
// rows keeping the row above, the row itself and PF rows below in registers, so every element of
// X is read from memory once per tile (plus the two halo rows of the tile).  Horizontal neighbours
// come from the neighbouring lane by shuffle, and at the band's two ends from one extra scalar
// load.  Before marching, the warp copies its receive segments -- the parts of the sections its
// device receives in this call (Eq. 1-2) that only this tile reads -- from the sender's buffer into
// its own; __syncwarp then orders those stores before the march reads them.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hda {

template <int DT>
struct Elem;
template <>
struct Elem<DT_F64> {
    using E = double;   // storage
    using A = double;   // arithmetic
    using V = double2;  // 16-byte chunk
    static constexpr int VEC = 2;
    __device__ static void unpack(const V &v, A *a) { a[0] = v.x; a[1] = v.y; }
    __device__ static V pack(const A *a) { return make_double2(a[0], a[1]); }
    __device__ static A load1(const E *p) { return *p; }
    __device__ static void store1(E *p, A a) { *p = a; }
};
template <>
struct Elem<DT_F32> {
    using E = float;
    using A = float;
    using V = float4;
    static constexpr int VEC = 4;
    __device__ static void unpack(const V &v, A *a) { a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w; }
    __device__ static V pack(const A *a) { return make_float4(a[0], a[1], a[2], a[3]); }
    __device__ static A load1(const E *p) { return *p; }
    __device__ static void store1(E *p, A a) { *p = a; }
};
template <>
struct Elem<DT_BF16> {
    using E = __nv_bfloat16;
    using A = float;
    using V = uint4;
    static constexpr int VEC = 8;
    __device__ static void unpack(const V &v, A *a)
    {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            a[2 * i] = __uint_as_float(w[i] << 16);
            a[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    __device__ static uint32_t bits(A a) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)); }
    __device__ static V pack(const A *a)
    {
        V v;
        v.x = bits(a[0]) | (bits(a[1]) << 16);
        v.y = bits(a[2]) | (bits(a[3]) << 16);
        v.z = bits(a[4]) | (bits(a[5]) << 16);
        v.w = bits(a[6]) | (bits(a[7]) << 16);
        return v;
    }
    __device__ static A load1(const E *p) { return __bfloat162float(*p); }
    __device__ static void store1(E *p, A a) { *p = __float2bfloat16_rn(a); }
};

// One row of a tile in registers: the lane's chunk plus the band's two edge elements (only
// meaningful on lane 0 / lane 31).
template <int DT>
struct Row {
    typename Elem<DT>::A v[Elem<DT>::VEC];
    typename Elem<DT>::A l, r;
};

template <int DT>
__device__ __forceinline__ void load_row(Row<DT> &row, const typename Elem<DT>::E *xrow, int x,
                                         bool act, bool needL, bool needR, int lane)
{
    using EL = Elem<DT>;
    if (act) {
        typename EL::V v = *reinterpret_cast<const typename EL::V *>(xrow + x);
        EL::unpack(v, row.v);
    }
    if (lane == 0 && needL) row.l = EL::load1(xrow + x - 1);
    if (lane == 31 && needR) row.r = EL::load1(xrow + x + EL::VEC);
}

template <int DT, int PF>
__global__ void __launch_bounds__(256) k_jacobi2d(const StenPart2D *__restrict__ parts,
                                                  const StenTile2D *__restrict__ tiles, int ntiles,
                                                  const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    constexpr int VEC = EL::VEC;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= ntiles) return;  // warp-uniform
    const StenTile2D t = tiles[wid];
    const StenPart2D P = parts[t.part];

    // receive: this tile's share of the device's incoming sections
    for (int s = 0; s < t.nseg; s++) {
        const Seg g = segs[t.seg0 + s];
        const E *src = reinterpret_cast<const E *>(g.src);
        E *dst = reinterpret_cast<E *>(g.dst);
        for (int k = lane; k < g.n; k += 32) dst[k * g.ds] = src[k * g.ss];
    }
    __syncwarp();

    const int x = t.cb + lane * VEC;
    const bool act = (x < t.c1 + 1) && (x + VEC > t.c0 - 1);
    const bool needL = (t.cb >= t.c0) && (t.cb < t.c1);
    const bool needR = (t.cb + 32 * VEC - 1 >= t.c0) && (t.cb + 32 * VEC - 1 < t.c1);
    const E *X = reinterpret_cast<const E *>(P.x) + (x - P.xlo1);
    E *Y = reinterpret_cast<E *>(P.y) + (x - P.ylo1);
    const int64_t xs = P.xs, ys = P.ys;

    Row<DT> up, mid, q[PF];
    load_row<DT>(up, X + (t.r0 - 1 - P.xlo0) * xs, 0, act, false, false, lane);
    load_row<DT>(mid, X + (t.r0 - P.xlo0) * xs, 0, act, needL, needR, lane);
#pragma unroll
    for (int k = 0; k < PF; k++)
        if (t.r0 + 1 + k <= t.r1) load_row<DT>(q[k], X + (t.r0 + 1 + k - P.xlo0) * xs, 0, act, needL, needR, lane);

    const bool full = (x >= t.c0) && (x + VEC <= t.c1);
    for (int r = t.r0; r < t.r1; r++) {
        const Row<DT> &dn = q[0];
        A left = __shfl_up_sync(0xffffffffu, mid.v[VEC - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, mid.v[0], 1);
        if (lane == 0) left = mid.l;
        if (lane == 31) right = mid.r;
        A out[VEC];
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const A w = k > 0 ? mid.v[k - 1] : left;
            const A e = k < VEC - 1 ? mid.v[k + 1] : right;
            A s = w + e;
            s = s + up.v[k];
            s = s + dn.v[k];
            out[k] = s * A(0.25);
        }
        E *yrow = Y + (r - P.ylo0) * ys;
        if (full) {
            *reinterpret_cast<typename EL::V *>(yrow) = EL::pack(out);
        } else if (act) {
#pragma unroll
            for (int k = 0; k < VEC; k++)
                if (x + k >= t.c0 && x + k < t.c1) EL::store1(yrow + k, out[k]);
        }
        up = mid;
        mid = q[0];
#pragma unroll
        for (int k = 0; k < PF - 1; k++) q[k] = q[k + 1];
        const int nr = r + 1 + PF;
        if (nr <= t.r1) load_row<DT>(q[PF - 1], X + (nr - P.xlo0) * xs, 0, act, needL, needR, lane);
    }
}

cudaError_t launch_jacobi2d(int dtype, const StenPart2D *parts, const StenTile2D *tiles,
                            int ntiles, const Seg *segs, int warps_per_cta, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (warps_per_cta < 1 || warps_per_cta > 8) warps_per_cta = 4;
    const int grid = (ntiles + warps_per_cta - 1) / warps_per_cta;
    const int block = 32 * warps_per_cta;
    switch (dtype) {
    case DT_F64: k_jacobi2d<DT_F64, 4><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_F32: k_jacobi2d<DT_F32, 4><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_BF16: k_jacobi2d<DT_BF16, 4><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// R = (X - Y)^2 in binary64 (a residual field for HDArrayReduce).
// ------------------------------------------------------------------------------------------
template <int DT>
__device__ __forceinline__ double ld64(const void *p, int64_t i)
{
    return (double)Elem<DT>::load1(reinterpret_cast<const typename Elem<DT>::E *>(p) + i);
}

template <int DT>
__global__ void __launch_bounds__(256) k_sqdiff(const PwTask *__restrict__ tasks)
{
    const PwTask t = tasks[blockIdx.x];
    const int nrows = t.row_end - t.row_begin;
    const int64_t total = (int64_t)nrows * t.n_inner;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int rr = (int)(i / t.n_inner), c = (int)(i - (int64_t)rr * t.n_inner);
        const int row = t.row_begin + rr;
        const int o = row / t.n_mid, m = row - o * t.n_mid;
        const double a = ld64<DT>(t.x, o * t.xs_outer + m * t.xs_mid + c);
        const double b = ld64<DT>(t.y, o * t.ys_outer + m * t.ys_mid + c);
        const double d = a - b;
        t.r[o * t.rs_outer + m * t.rs_mid + c] = d * d;
    }
}

cudaError_t launch_sqdiff(int dtype, const PwTask *tasks, int ntasks, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    switch (dtype) {
    case DT_F64: k_sqdiff<DT_F64><<<ntasks, 256, 0, s>>>(tasks); break;
    case DT_F32: k_sqdiff<DT_F32><<<ntasks, 256, 0, s>>>(tasks); break;
    case DT_BF16: k_sqdiff<DT_BF16><<<ntasks, 256, 0, s>>>(tasks); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hda
