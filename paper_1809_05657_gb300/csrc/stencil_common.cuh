// stencil_common.cuh -- storage types, register rows and the receive phase shared by the fused
// stencil kernels (k_stencil2d.cu, k_stencil3d.cu).
#pragma once

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
    // two values rounded to nearest even into one bfloat16 pair (the first in the low half, as
    // stored), one conversion instruction per pair
    __device__ static uint32_t pair(A lo, A hi)
    {
        const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t *>(&p);
    }
    __device__ static V pack(const A *a)
    {
        V v;
        v.x = pair(a[0], a[1]);
        v.y = pair(a[2], a[3]);
        v.z = pair(a[4], a[5]);
        v.w = pair(a[6], a[7]);
        return v;
    }
    __device__ static A load1(const E *p) { return __bfloat162float(*p); }
    __device__ static void store1(E *p, A a) { *p = __float2bfloat16_rn(a); }
};

// Copy elements [first, total) step `stride` of a tile's receive segments (sender buffer -> own
// buffer), all segments flattened into one index space and four element copies in flight per
// thread, so a tile with several small faces pays about one memory round trip, not one per face.
template <typename E>
__device__ __forceinline__ void receive_flat(const Seg *__restrict__ segs, int seg0, int nseg, int first, int stride)
{
    // segments in order; this thread's elements of each segment in batches of four loads, then
    // four stores, and the batch carries over from one segment into the next
    E v[4];
    E *dst[4];
    int nb = 0;
    for (int s = 0; s < nseg; s++) {
        const Seg g = segs[seg0 + s];
        const int total = g.n * g.m;
        const E *src = reinterpret_cast<const E *>(g.src);
        E *d0 = reinterpret_cast<E *>(g.dst);
        int o = first / g.n, k = first - (first / g.n) * g.n;
        const int dof = stride / g.n, dk = stride - dof * g.n;
        for (int i = first; i < total; i += stride) {
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (u == nb) {
                    v[u] = src[o * g.sso + k * g.ss];
                    dst[u] = d0 + o * g.dso + k * g.ds;
                }
            if (++nb == 4) {
#pragma unroll
                for (int u = 0; u < 4; u++) *dst[u] = v[u];
                nb = 0;
            }
            o += dof;
            k += dk;
            if (k >= g.n) {
                k -= g.n;
                o += 1;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
        if (u < nb) *dst[u] = v[u];
}

// A receive segment whose rows are contiguous runs at the same 16-byte phase in the sender's and
// the receiver's buffer (row faces in 2-D, y and z faces in 3-D): h0 elements up to the first
// 16-byte boundary, then nc whole 16-byte chunks, then the tail.  nc = 0: copied element-wise.
template <typename E>
__device__ __forceinline__ void run_split(const Seg &g, int &h0, int &nc)
{
    constexpr int VEC = 16 / (int)sizeof(E);
    h0 = 0;
    nc = 0;
    const uintptr_t sa = reinterpret_cast<uintptr_t>(g.src), da = reinterpret_cast<uintptr_t>(g.dst);
    if (g.ss != 1 || g.ds != 1 || g.n < 2 * VEC || ((sa ^ da) & 15) != 0) return;
    if (g.m > 1 && ((((int64_t)sizeof(E) * g.sso) & 15) != 0 || (((int64_t)sizeof(E) * g.dso) & 15) != 0)) return;
    h0 = (int)(((16 - (sa & 15)) & 15) / sizeof(E));
    nc = (g.n - h0) / VEC;
}

// The same copy for a whole CTA, with the contiguous runs moved in 16-byte chunks: this thread's
// share of items first, first + stride, ... of every segment, first the chunks of the contiguous
// runs, then the remaining elements, each pass with four copies in flight per thread.  (The warp
// kernels keep the element-wise form: the chunk pass costs them registers in their march.)
template <typename E>
__device__ __forceinline__ void receive_flat_vec(const Seg *__restrict__ segs, int seg0, int nseg, int first, int stride)
{
    constexpr int VEC = 16 / (int)sizeof(E);
    {  // 16-byte chunks
        uint4 v[4];
        uint4 *dst[4];
        int nb = 0;
        for (int s = 0; s < nseg; s++) {
            const Seg g = segs[seg0 + s];
            int h0, nc;
            run_split<E>(g, h0, nc);
            if (nc == 0) continue;
            const int total = nc * g.m;
            const E *src = reinterpret_cast<const E *>(g.src) + h0;
            E *d0 = reinterpret_cast<E *>(g.dst) + h0;
            int o = first / nc, c = first - (first / nc) * nc;
            const int dof = stride / nc, dc = stride - dof * nc;
            for (int i = first; i < total; i += stride) {
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u == nb) {
                        v[u] = *reinterpret_cast<const uint4 *>(src + o * g.sso + c * VEC);
                        dst[u] = reinterpret_cast<uint4 *>(d0 + o * g.dso + c * VEC);
                    }
                if (++nb == 4) {
#pragma unroll
                    for (int u = 0; u < 4; u++) *dst[u] = v[u];
                    nb = 0;
                }
                o += dof;
                c += dc;
                if (c >= nc) {
                    c -= nc;
                    o += 1;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (u < nb) *dst[u] = v[u];
    }
    {  // elements: whole segments that are not contiguous runs, heads and tails of those that are
        E v[4];
        E *dst[4];
        int nb = 0;
        for (int s = 0; s < nseg; s++) {
            const Seg g = segs[seg0 + s];
            int h0, nc;
            run_split<E>(g, h0, nc);
            const int per = g.n - nc * VEC;  // elements per row left to this pass
            if (per == 0) continue;
            const int skip = nc * VEC;       // element q of a row's share is element q (< h0) or q + skip
            const int total = per * g.m;
            const E *src = reinterpret_cast<const E *>(g.src);
            E *d0 = reinterpret_cast<E *>(g.dst);
            int o = first / per, q = first - (first / per) * per;
            const int dof = stride / per, dq = stride - dof * per;
            for (int i = first; i < total; i += stride) {
                const int k = q < h0 ? q : q + skip;
#pragma unroll
                for (int u = 0; u < 4; u++)
                    if (u == nb) {
                        v[u] = src[o * g.sso + k * g.ss];
                        dst[u] = d0 + o * g.dso + k * g.ds;
                    }
                if (++nb == 4) {
#pragma unroll
                    for (int u = 0; u < 4; u++) *dst[u] = v[u];
                    nb = 0;
                }
                o += dof;
                q += dq;
                if (q >= per) {
                    q -= per;
                    o += 1;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (u < nb) *dst[u] = v[u];
    }
}

// The warp's receive phase, then __syncwarp orders the copies before the warp's loads: the
// barrier orders memory among the threads that take part in it, and cp.async reads are memory
// operations of the issuing thread, so they see the other lanes' stores.
template <typename E>
__device__ __forceinline__ void receive_segments(const Seg *__restrict__ segs, int seg0, int nseg, int lane)
{
    if (nseg > 0) receive_flat<E>(segs, seg0, nseg, lane, 32);
    __syncwarp();
}

// One row of a tile in registers: the lane's chunk plus the band's two edge elements (only
// meaningful on lane 0 / lane 31).
template <int DT>
struct Row {
    typename Elem<DT>::A v[Elem<DT>::VEC];
    typename Elem<DT>::A l, r;
};

// FILL: lanes past the band's end hold ones (their results are not stored, but they take part in
// the warp's vote on the division path, which a sum of ones keeps on the fast side).
template <int DT, bool FILL = false>
__device__ __forceinline__ void load_row(Row<DT> &row, const typename Elem<DT>::E *xrow, int x,
                                         bool act, bool needL, bool needR, int lane)
{
    using EL = Elem<DT>;
    if (act) {
        typename EL::V v = *reinterpret_cast<const typename EL::V *>(xrow + x);
        EL::unpack(v, row.v);
    } else if (FILL) {
#pragma unroll
        for (int k = 0; k < EL::VEC; k++) row.v[k] = typename EL::A(1);
    }
    if (lane == 0 && needL) row.l = EL::load1(xrow + x - 1);
    if (lane == 31 && needR) row.r = EL::load1(xrow + x + EL::VEC);
}

// Correctly rounded s / 6 in binary32 without a division: q = RN(s * c) with c = RN(1/6), the
// remainder r = s - q * 6 (exact with one FMA), then q + r * c rounded once -- the correction step
// for division by a constant known in advance (Brisebarre, Muller & Raina, IEEE Trans. Computers
// 53(8), 2004).  Checked against IEEE division for every finite binary32 input: identical whenever
// 2^-100 <= |s|.  Zero, tiny, infinite and NaN sums take the true division instead (the bare steps
// give +0 for -0 and NaN for an infinity).
__device__ __forceinline__ float div6_fast(float s)
{
    const float c = 0x1.555556p-3f;  // RN(1/6)
    const float q = __fmul_rn(s, c);
    const float r = __fmaf_rn(-q, 6.0f, s);
    return __fmaf_rn(r, c, q);
}
// 2^-100 <= |s| <= FLT_MAX, as one unsigned range test on the magnitude's bits
__device__ __forceinline__ bool div6_fast_ok(float s)
{
    return (__float_as_uint(s) & 0x7fffffffu) - 0x0d800000u <= 0x71ffffffu;
}

// s[k] / 6 for every k, in place, correctly rounded.  The rare sums outside the fast method's range
// send the lanes executing together (one vote over __activemask) through IEEE division, so the
// common path carries no division instructions.
template <int N>
__device__ __forceinline__ void div6_n(float (&s)[N])
{
    bool slow = false;
#pragma unroll
    for (int k = 0; k < N; k++) slow |= !div6_fast_ok(s[k]);
    if (__any_sync(__activemask(), slow)) {
#pragma unroll
        for (int k = 0; k < N; k++) s[k] = __fdiv_rn(s[k], 6.0f);
    } else {
#pragma unroll
        for (int k = 0; k < N; k++) s[k] = div6_fast(s[k]);
    }
}
template <int N>
__device__ __forceinline__ void div6_n(double (&s)[N])
{
#pragma unroll
    for (int k = 0; k < N; k++) s[k] = s[k] / 6.0;
}

// Transaction-count mbarriers for bulk tensor copies: a non-blocking probe of a phase, and a wait
// that gives up after `limit` probes (the caller reports the failure instead of hanging).
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

constexpr unsigned TMA_DRAIN_LIMIT = 1u << 22;  // polls when draining after a failed wait

// Asynchronous global -> shared copies (cp.async) and their group waits.
__device__ __forceinline__ void cpa16(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa8(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa4(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Edge element copy: the smallest cp.async is 4 bytes, so a bfloat16 edge travels as the aligned
// 4-byte pair that contains it.
template <int DT>
__device__ __forceinline__ void edge_copy(uint32_t saddr, const typename Elem<DT>::E *g, bool left)
{
    if (sizeof(typename Elem<DT>::E) == 8) cpa8(saddr, g);
    else if (sizeof(typename Elem<DT>::E) == 4) cpa4(saddr, g);
    else cpa4(saddr, left ? (const void *)(g - 1) : (const void *)g);
}
template <int DT>
__device__ __forceinline__ typename Elem<DT>::A edge_read(const uint4 *slot, bool left)
{
    using A = typename Elem<DT>::A;
    if (sizeof(typename Elem<DT>::E) == 8) return (A) * reinterpret_cast<const double *>(slot);
    if (sizeof(typename Elem<DT>::E) == 4) return (A) * reinterpret_cast<const float *>(slot);
    const uint32_t w = *reinterpret_cast<const uint32_t *>(slot);
    return (A)__uint_as_float(left ? (w & 0xffff0000u) : (w << 16));
}


// Receive segments copied by a whole CTA, then a barrier orders them before the CTA's loads (as
// for the warp form above, at CTA scope).  RUNS: contiguous runs in 16-byte chunks (measured
// faster for the 3-D and binary32/binary64 2-D CTA kernels; the bfloat16 2-D kernel keeps the
// element form, whose registers fit its march better).
template <typename E, bool RUNS = true>
__device__ __forceinline__ void receive_segments_cta(const Seg *__restrict__ segs, int seg0, int nseg)
{
    if (nseg > 0) {
        if (RUNS) receive_flat_vec<E>(segs, seg0, nseg, threadIdx.x, blockDim.x);
        else receive_flat<E>(segs, seg0, nseg, threadIdx.x, blockDim.x);
    }
    __syncthreads();
}

}  // namespace hda
