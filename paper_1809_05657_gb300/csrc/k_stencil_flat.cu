// k_stencil_flat.cu -- "flat block" forms of the fused stencil kernels for partitions whose shape
// fits the 32-lane x 16-byte bands badly (narrow, short or uneven work boxes).
//
// A CTA owns a block of the device's work box: rows [r0, r1) x columns [c0, c1) in 2-D, or rows
// [y0, y0+ny) x columns [x0, x1) of every plane z in [z0, z1) in 3-D.  The block and its one-element
// halo are staged in shared memory, and the 256 threads walk the block's cells in row-major order
// (consecutive threads, consecutive columns), so every thread has work whatever the block's width.
// 2-D: one load phase, one compute phase.  3-D: a ring of NS planes filled by 4- or 8-byte
// cp.async, marching z as in the banded kernel.  The arithmetic is the banded kernels' (same order,
// same rounding), and the receive phase is the same flattened copy.  binary32 and binary64.
#include "stencil_common.cuh"

namespace hda {

namespace {

// Walk `count` cells of a row-major (rows x w) block starting at thread index `t`, stepping by
// `step`, without dividing in the loop: f(row, col) for each.
template <typename F>
__device__ __forceinline__ void walk(int t, int step, int count, int w, F f)
{
    if (t >= count) return;
    int r = t / w, c = t - r * w;
    const int dr = step / w, dc = step - dr * w;
    for (int i = t; i < count; i += step) {
        f(r, c);
        r += dr;
        c += dc;
        if (c >= w) {
            c -= w;
            r += 1;
        }
    }
}

template <int DT>
__device__ __forceinline__ void cpa_elem(uint32_t saddr, const void *g)
{
    if (sizeof(typename Elem<DT>::E) == 8) cpa8(saddr, g);
    else cpa4(saddr, g);
}

}  // namespace

template <int DT>
__global__ void __launch_bounds__(256) k_jacobi2d_flat(const StenPart2D *__restrict__ parts,
                                                       const StenTile2D *__restrict__ tiles,
                                                       const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    extern __shared__ uint4 smem4[];
    E *sm = reinterpret_cast<E *>(smem4);
    const StenTile2D t = tiles[blockIdx.x];
    const StenPart2D P = parts[t.part];
    receive_segments_cta<E>(segs, t.seg0, t.nseg);
    const int R = t.r1 - t.r0, W = t.c1 - t.c0, SW = W + 2;
    const E *X = reinterpret_cast<const E *>(P.x);
    // stage rows r0-1 .. r1 and columns c0-1 .. c1 (the corners are loaded but not used)
    walk(threadIdx.x, blockDim.x, (R + 2) * SW, SW, [&](int rr, int cc) {
        sm[rr * SW + cc] = X[(int64_t)(t.r0 - 1 + rr - P.xlo0) * P.xs + (t.c0 - 1 + cc - P.xlo1)];
    });
    __syncthreads();
    E *Y = reinterpret_cast<E *>(P.y);
    walk(threadIdx.x, blockDim.x, R * W, W, [&](int r, int c) {
        const E *m = sm + (r + 1) * SW + (c + 1);
        A s = (A)m[-1] + (A)m[1];
        s = s + (A)m[-SW];
        s = s + (A)m[SW];
        Y[(int64_t)(t.r0 + r - P.ylo0) * P.ys + (t.c0 + c - P.ylo1)] = (E)(s * A(0.25));
    });
}

template <int DT, int NS>
__global__ void __launch_bounds__(256) k_stencil3d_flat(const StenPart3D *__restrict__ parts,
                                                        const StenTile3D *__restrict__ tiles,
                                                        const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    extern __shared__ uint4 smem4[];
    E *sm = reinterpret_cast<E *>(smem4);
    const StenTile3D t = tiles[blockIdx.x];
    const StenPart3D P = parts[t.part];
    receive_segments_cta<E>(segs, t.seg0, t.nseg);
    const int NY = t.ny, NX = t.x1 - t.x0, SX = NX + 2, PL = (NY + 2) * SX;  // one staged plane
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sm);
    const E *X = reinterpret_cast<const E *>(P.x);

    auto issue_plane = [&](int zp) {
        const int stage = (zp - t.z0 + 1) % NS;
        const E *pz = X + (int64_t)(zp - P.xlo0) * P.xs0;
        walk(threadIdx.x, blockDim.x, PL, SX, [&](int rr, int cc) {
            const E *g = pz + (int64_t)(t.y - 1 + rr - P.xlo1) * P.xs1 + (t.x0 - 1 + cc - P.xlo2);
            cpa_elem<DT>(sbase + (uint32_t)(stage * PL + rr * SX + cc) * (uint32_t)sizeof(E), g);
        });
    };
#pragma unroll 1
    for (int k = 0; k < NS - 1; k++) {
        const int zp = t.z0 - 1 + k;
        if (zp <= t.z1) issue_plane(zp);
        cpa_commit();
    }
    E *Y = reinterpret_cast<E *>(P.y);
    for (int z = t.z0; z < t.z1; z++) {
        cpa_wait<NS - 4>();
        __syncthreads();
        if (z - 2 + NS <= t.z1) issue_plane(z - 2 + NS);
        cpa_commit();
        const E *s0 = sm + ((z - t.z0 + 1) % NS) * PL;
        const E *sm1 = sm + ((z - t.z0) % NS) * PL;
        const E *sp1 = sm + ((z - t.z0 + 2) % NS) * PL;
        E *yz = Y + (int64_t)(z - P.ylo0) * P.ys0;
        walk(threadIdx.x, blockDim.x, NY * NX, NX, [&](int r, int c) {
            const int o = (r + 1) * SX + (c + 1);
            A s = (A)s0[o - 1] + (A)s0[o + 1];
            s = s + (A)s0[o - SX];
            s = s + (A)s0[o + SX];
            s = s + (A)sm1[o];
            s = s + (A)sp1[o];
            A q[1] = {s};
            div6_n(q);
            yz[(int64_t)(t.y + r - P.ylo1) * P.ys1 + (t.x0 + c - P.ylo2)] = (E)q[0];
        });
    }
    cpa_wait<0>();
}

size_t flat2d_smem(int dtype, int rows, int cols)
{
    return (size_t)(rows + 2) * (cols + 2) * (dtype == DT_F64 ? 8 : 4);
}

size_t flat3d_smem(int dtype, int ny, int nx)
{
    return (size_t)FLAT3D_STAGES * (ny + 2) * (nx + 2) * (dtype == DT_F64 ? 8 : 4);
}

cudaError_t launch_jacobi2d_flat(int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                 const Seg *segs, size_t smem, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    static bool attr[2] = {false, false};
    const int which = dtype == DT_F64 ? 0 : 1;
    if (!attr[which]) {
        cudaError_t e = which == 0
            ? cudaFuncSetAttribute(k_jacobi2d_flat<DT_F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
            : cudaFuncSetAttribute(k_jacobi2d_flat<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr[which] = true;
    }
    if (dtype == DT_F64) k_jacobi2d_flat<DT_F64><<<ntiles, 256, smem, s>>>(parts, tiles, segs);
    else if (dtype == DT_F32) k_jacobi2d_flat<DT_F32><<<ntiles, 256, smem, s>>>(parts, tiles, segs);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_stencil3d_flat(int dtype, const StenPart3D *parts, const StenTile3D *tiles, int ntiles,
                                  const Seg *segs, size_t smem, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    static bool attr[2] = {false, false};
    const int which = dtype == DT_F64 ? 0 : 1;
    if (!attr[which]) {
        cudaError_t e = which == 0
            ? cudaFuncSetAttribute(k_stencil3d_flat<DT_F64, FLAT3D_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024)
            : cudaFuncSetAttribute(k_stencil3d_flat<DT_F32, FLAT3D_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr[which] = true;
    }
    if (dtype == DT_F64) k_stencil3d_flat<DT_F64, FLAT3D_STAGES><<<ntiles, 256, smem, s>>>(parts, tiles, segs);
    else if (dtype == DT_F32) k_stencil3d_flat<DT_F32, FLAT3D_STAGES><<<ntiles, 256, smem, s>>>(parts, tiles, segs);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace hda
