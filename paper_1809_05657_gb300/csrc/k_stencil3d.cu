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
            out[k] = div6(s);
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

// ------------------------------------------------------------------------------------------
// CTA variant: one CTA per tile of ny <= 8 consecutive rows (one warp each) of one band, marching
// z.  Plane z' of rows y0-1 .. y0+ny (the tile's rows and their y neighbours) goes into stage
// (z' - z0 + 1) % NS of a shared-memory ring by cp.async from every thread, so each input row
// is fetched once per CTA and NS - 4 planes are in flight ahead of the one being computed.  At step
// z the CTA reads planes z-1, z, z+1 and refills the stage of plane z-2 (read by nobody since the
// barrier of this step).  Stage layout: (8 + 2) rows x (32 chunks + 2 edge slots) x 16 bytes.
// ------------------------------------------------------------------------------------------
template <int DT, int NS>
__global__ void __launch_bounds__(256, 4) k_stencil3d_cta(const StenPart3D *__restrict__ parts,
                                                       const StenTile3D *__restrict__ tiles,
                                                       const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    constexpr int VEC = EL::VEC;
    constexpr int ROWS = 10, SLOTS = 34, STAGE = ROWS * SLOTS;  // in 16-byte slots
    extern __shared__ uint4 smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const StenTile3D t = tiles[blockIdx.x];
    const StenPart3D P = parts[t.part];
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(smem);

    receive_segments_cta<E>(segs, t.seg0, t.nseg);

    const int ny = t.ny;
    const int64_t zs = P.xs0, ys = P.xs1;
    // row rr (0 .. ny+1) of the staged planes is array row y0 - 1 + rr
    const E *xbase = reinterpret_cast<const E *>(P.x) + (int64_t)(t.y - 1 - P.xlo1) * ys + (t.xb - P.xlo2);
    const int nrows = ny + 2;
    const bool needL = (t.xb >= t.x0) && (t.xb < t.x1);
    const bool needR = (t.xb + 32 * VEC - 1 >= t.x0) && (t.xb + 32 * VEC - 1 < t.x1);

    // This thread's share of every staged plane, fixed for the whole march: at most two 16-byte
    // chunks (rows x 32 chunks over 256 threads) and possibly one band-end edge element.
    const int nitems = nrows * 32;  // <= 320: thread t copies items t and t + 256
    const int ch = threadIdx.x & 31, xc = t.xb + ch * VEC;
    const bool chunk_ok = xc < t.x1 + 1 && xc + VEC > t.x0 - 1;
    const int rr0 = threadIdx.x >> 5, rr1 = rr0 + 8;
    const bool has0 = chunk_ok && threadIdx.x < nitems;
    const bool has1 = chunk_ok && threadIdx.x + 256 < nitems;
    const int64_t g0 = (int64_t)rr0 * ys + ch * VEC, g1 = (int64_t)rr1 * ys + ch * VEC;
    const uint32_t so0 = (uint32_t)(rr0 * SLOTS + ch) * 16u, so1 = (uint32_t)(rr1 * SLOTS + ch) * 16u;
    const int q = threadIdx.x;
    const bool eL = q < ny && needL, eR = q >= 32 && q < 32 + ny && needR;
    const int erow = eL ? q + 1 : q - 32 + 1;
    const int64_t eoff = (int64_t)erow * ys + (eL ? -1 : 32 * VEC);
    const uint32_t esoff = (uint32_t)(erow * SLOTS + (eL ? 32 : 33)) * 16u;
    auto issue_plane = [&](int zp) {
        const int stage = (zp - t.z0 + 1) % NS;
        const uint32_t sb = ring_s + (uint32_t)(stage * STAGE) * 16u;
        const E *pz = xbase + (int64_t)(zp - P.xlo0) * zs;
        if (has0) cpa16(sb + so0, pz + g0);
        if (has1) cpa16(sb + so1, pz + g1);
        if (eL || eR) edge_copy<DT>(sb + esoff, pz + eoff, eL);
    };

    // prologue: planes z0-1 .. z0+NS-3
#pragma unroll 1
    for (int k = 0; k < NS - 1; k++) {
        const int zp = t.z0 - 1 + k;
        if (zp <= t.z1) issue_plane(zp);
        cpa_commit();
    }
    const int x = t.xb + lane * VEC;
    const bool act = (x < t.x1 + 1) && (x + VEC > t.x0 - 1);
    const bool full = (x >= t.x0) && (x + VEC <= t.x1);
    const bool mine = w < ny;
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.y + w - P.ylo1) * P.ys1 + (x - P.ylo2) +
            (int64_t)(t.z0 - P.ylo0) * P.ys0;
    for (int z = t.z0; z < t.z1; z++) {
        cpa_wait<NS - 4>();  // planes up to z + 1 have landed (this thread's copies)
        __syncthreads();     // ... and every other thread's
        if (z - 2 + NS <= t.z1) issue_plane(z - 2 + NS);
        cpa_commit();
        if (mine) {
            const int k0 = z - t.z0;
            const uint4 *sm1 = smem + (k0 % NS) * STAGE;
            const uint4 *s0 = smem + ((k0 + 1) % NS) * STAGE;
            const uint4 *sp1 = smem + ((k0 + 2) % NS) * STAGE;
            const int me = w + 1;  // my row in the staged planes
            Row<DT> c, ym, yp1, zm, zp;
            if (act) {
                EL::unpack(*reinterpret_cast<const typename EL::V *>(s0 + me * SLOTS + lane), c.v);
                EL::unpack(*reinterpret_cast<const typename EL::V *>(s0 + (me - 1) * SLOTS + lane), ym.v);
                EL::unpack(*reinterpret_cast<const typename EL::V *>(s0 + (me + 1) * SLOTS + lane), yp1.v);
                EL::unpack(*reinterpret_cast<const typename EL::V *>(sm1 + me * SLOTS + lane), zm.v);
                EL::unpack(*reinterpret_cast<const typename EL::V *>(sp1 + me * SLOTS + lane), zp.v);
            }
            A left = __shfl_up_sync(0xffffffffu, c.v[VEC - 1], 1);
            A right = __shfl_down_sync(0xffffffffu, c.v[0], 1);
            if (lane == 0 && needL) left = edge_read<DT>(s0 + me * SLOTS + 32, true);
            if (lane == 31 && needR) right = edge_read<DT>(s0 + me * SLOTS + 33, false);
            A out[VEC];
#pragma unroll
            for (int k = 0; k < VEC; k++) {
                const A wv = k > 0 ? c.v[k - 1] : left;
                const A ev = k < VEC - 1 ? c.v[k + 1] : right;
                A s = wv + ev;
                s = s + ym.v[k];
                s = s + yp1.v[k];
                s = s + zm.v[k];
                s = s + zp.v[k];
                out[k] = div6(s);
            }
            if (full) {
                *reinterpret_cast<typename EL::V *>(yp) = EL::pack(out);
            } else if (act) {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (x + k >= t.x0 && x + k < t.x1) EL::store1(yp + k, out[k]);
            }
        }
        yp += P.ys0;
    }
    cpa_wait<0>();
}

cudaError_t launch_stencil3d(int dtype, const StenPart3D *parts, const StenTile3D *tiles,
                             int ntiles, const Seg *segs, int warps_per_cta, int variant, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (variant == 1) {
        constexpr int NS = 8;
        const size_t sm = (size_t)NS * 10 * 34 * 16;
        switch (dtype) {
        case DT_F64: k_stencil3d_cta<DT_F64, NS><<<ntiles, 256, sm, s>>>(parts, tiles, segs); break;
        case DT_F32: k_stencil3d_cta<DT_F32, NS><<<ntiles, 256, sm, s>>>(parts, tiles, segs); break;
        case DT_BF16: k_stencil3d_cta<DT_BF16, NS><<<ntiles, 256, sm, s>>>(parts, tiles, segs); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
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
