// k_stencil3d.cu -- the 3-D 7-point analogue of the Jacobi step on every logical device's work
// box, fused with the exchange:
//
//   Y[z][y][x] = (X[z][y][x-1] + X[z][y][x+1] + X[z][y-1][x] + X[z][y+1][x]
//                 + X[z-1][y][x] + X[z+1][y][x]) / 6
//
// summed left to right in that order, one correctly rounded division, in the storage precision
// (bfloat16 storage: binary32 arithmetic, round to nearest even on the store).
//
// One warp per tile: a row y, a band of 32 lanes x one 16-byte chunk, marching z through
// [z0, z1).  The rows (z-1, y), (z, y) and PF planes ahead stay in registers; the rows y-1 and
// y+1 of the current plane are loaded one plane ahead (consecutive warps of a CTA hold consecutive
// rows, so those loads mostly hit L1); x neighbours come by shuffle and, at the band ends, from
// one scalar load.  The tile first copies its receive segments (the parts of its device's incoming
// faces that only it reads) from the senders' buffers, as in the 2-D kernel.
#include "stencil_common.cuh"

namespace hda {

template <int DT, int PF>
__global__ void __launch_bounds__(256) k_stencil3d(const StenPart3D *__restrict__ parts,
                                                   const StenTile3D *__restrict__ tiles, int ntiles,
                                                   const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    constexpr int VEC = EL::VEC;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= ntiles) return;  // warp-uniform
    const StenTile3D t = tiles[wid];
    const StenPart3D P = parts[t.part];

    receive_segments<E>(segs, t.seg0, t.nseg, lane);

    const int x = t.xb + lane * VEC;
    const bool act = (x < t.x1 + 1) && (x + VEC > t.x0 - 1);
    const bool needL = (t.xb >= t.x0) && (t.xb < t.x1);
    const bool needR = (t.xb + 32 * VEC - 1 >= t.x0) && (t.xb + 32 * VEC - 1 < t.x1);
    const int64_t zs = P.xs0, zsy = P.ys0;
    const E *Xc = reinterpret_cast<const E *>(P.x) + (t.y - P.xlo1) * P.xs1 + (x - P.xlo2);
    const E *Xm = Xc - P.xs1;
    const E *Xp = Xc + P.xs1;
    E *Yc = reinterpret_cast<E *>(P.y) + (t.y - P.ylo1) * P.ys1 + (x - P.ylo2);
    const int zx = (int)P.xlo0, zy = (int)P.ylo0;  // buffer origins along z

    Row<DT> zm, zc, q[PF], ym, yp, nym, nyp;
    load_row<DT>(zm, Xc + (int64_t)(t.z0 - 1 - zx) * zs, 0, act, false, false, lane);
    load_row<DT>(zc, Xc + (int64_t)(t.z0 - zx) * zs, 0, act, needL, needR, lane);
#pragma unroll
    for (int k = 0; k < PF; k++)
        if (t.z0 + 1 + k <= t.z1) load_row<DT>(q[k], Xc + (int64_t)(t.z0 + 1 + k - zx) * zs, 0, act, needL, needR, lane);
    load_row<DT>(ym, Xm + (int64_t)(t.z0 - zx) * zs, 0, act, false, false, lane);
    load_row<DT>(yp, Xp + (int64_t)(t.z0 - zx) * zs, 0, act, false, false, lane);

    const bool full = (x >= t.x0) && (x + VEC <= t.x1);
    for (int z = t.z0; z < t.z1; z++) {
        if (z + 1 < t.z1) {
            load_row<DT>(nym, Xm + (int64_t)(z + 1 - zx) * zs, 0, act, false, false, lane);
            load_row<DT>(nyp, Xp + (int64_t)(z + 1 - zx) * zs, 0, act, false, false, lane);
        }
        A left = __shfl_up_sync(0xffffffffu, zc.v[VEC - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, zc.v[0], 1);
        if (lane == 0) left = zc.l;
        if (lane == 31) right = zc.r;
        A out[VEC];
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const A w = k > 0 ? zc.v[k - 1] : left;
            const A e = k < VEC - 1 ? zc.v[k + 1] : right;
            A s = w + e;
            s = s + ym.v[k];
            s = s + yp.v[k];
            s = s + zm.v[k];
            s = s + q[0].v[k];
            out[k] = s / A(6);
        }
        E *yrow = Yc + (int64_t)(z - zy) * zsy;
        if (full) {
            *reinterpret_cast<typename EL::V *>(yrow) = EL::pack(out);
        } else if (act) {
#pragma unroll
            for (int k = 0; k < VEC; k++)
                if (x + k >= t.x0 && x + k < t.x1) EL::store1(yrow + k, out[k]);
        }
        zm = zc;
        zc = q[0];
#pragma unroll
        for (int k = 0; k < PF - 1; k++) q[k] = q[k + 1];
        const int nz = z + 1 + PF;
        if (nz <= t.z1) load_row<DT>(q[PF - 1], Xc + (int64_t)(nz - zx) * zs, 0, act, needL, needR, lane);
        ym = nym;
        yp = nyp;
    }
}

cudaError_t launch_stencil3d(int dtype, const StenPart3D *parts, const StenTile3D *tiles,
                             int ntiles, const Seg *segs, int warps_per_cta, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (warps_per_cta < 1 || warps_per_cta > 8) warps_per_cta = 8;
    const int grid = (ntiles + warps_per_cta - 1) / warps_per_cta;
    const int block = 32 * warps_per_cta;
    switch (dtype) {
    case DT_F64: k_stencil3d<DT_F64, 3><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_F32: k_stencil3d<DT_F32, 3><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_BF16: k_stencil3d<DT_BF16, 3><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hda
