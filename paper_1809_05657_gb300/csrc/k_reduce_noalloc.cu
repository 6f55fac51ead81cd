// k_reduce_noalloc.cu -- a reduction entry point that allocates no device memory.
//
// HDArrayReduce allocates its scratch (per-CTA partial sums, a completion counter) and its task
// table with cudaMalloc.  Some callers cannot allocate: code whose device memory is owned by
// another allocator (a framework's caching allocator that has reserved most of the GPU, where a
// direct cudaMalloc can fail or fragment the pool), and latency-critical paths on which the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.  For them,
// HDArrayReduceBufferNoAlloc reduces one strided box of an existing device buffer into a caller-
// provided device double, using scratch that lives in a fixed-size static device array of this
// file instead of allocated memory.
//
// The first call on each device looks up the array's device address (cudaGetSymbolAddress, with
// that device current) and remembers it; make that first call before any stream capture on the
// device.  The static array is loaded with the library on every GPU that uses it and stays there
// until the process exits.  Every call shares it and it keeps the last call's contents, so the completion
// counter is cleared (cudaMemsetAsync, no allocation) at the start of every call; calls that
// overlap on the GPU (on different streams, say) race on the shared scratch and must not overlap.
#include <cuda_bf16.h>
#include <string.h>

#include "hdarray.h"
#include "kernels.h"

namespace {

// The scratch holds one partial per CTA, so a call runs at most NOALLOC_MAX_PARTIALS CTAs.  A call
// reduces at most NOALLOC_MAX_ELEMS elements: the limit keeps one call's run time bounded (16 GiB
// of binary64 at most, a few milliseconds at HBM rate), so work queued behind it on the stream is
// not held up for long; larger boxes are reduced in pieces by the caller.  The scratch's size does
// not depend on the element count.
constexpr int NOALLOC_MAX_PARTIALS = 1024;
constexpr int64_t NOALLOC_MAX_ELEMS = (int64_t)1 << 31;
constexpr int64_t NOALLOC_SEG = 8192;  // elements of one work item (a row, or a piece of a long row)
constexpr int NOALLOC_COUNTER_OFFSET = NOALLOC_MAX_PARTIALS * 8;

// 8 KiB of partials, then the counter (zeroed before every call).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_COUNTER_OFFSET + 256];

// Host-side device address of g_noalloc_scratch, per device, from cudaGetSymbolAddress (the
// symbol's name in host code is only a stand-in, never a device address).
constexpr int MAX_DEVICES = 64;
unsigned char *g_scratch_addr[MAX_DEVICES] = {nullptr};

template <int DT>
__device__ __forceinline__ double ld(const void *p, int64_t i);
template <>
__device__ __forceinline__ double ld<hda::DT_F64>(const void *p, int64_t i) { return reinterpret_cast<const double *>(p)[i]; }
template <>
__device__ __forceinline__ double ld<hda::DT_F32>(const void *p, int64_t i) { return (double)reinterpret_cast<const float *>(p)[i]; }
template <>
__device__ __forceinline__ double ld<hda::DT_BF16>(const void *p, int64_t i)
{
    return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}

template <int OP>
__device__ __forceinline__ double fold(double a, double b)
{
    if (OP == 0) return a + b;
    if (OP == 1) return a * b;
    if (OP == 2) return b > a ? b : a;
    return b < a ? b : a;
}

// The box is cut into work items: each row of the box (a run of n_inner contiguous elements) is
// split into n_seg segments of at most NOALLOC_SEG elements, and the items (row, segment) are
// numbered row-major.  CTA b folds the contiguous item range [b*per, (b+1)*per): its warps take the
// items in turn and the lanes of a warp stride the segment, four independent loads in flight per
// lane.  A fixed shuffle / shared-memory tree gives the CTA's partial, and the last CTA to finish
// folds the partials in index order.  Item ranges, the fold order in each lane and the trees all
// depend on the box's shape only, so the result is deterministic.  A 1-D box or a box of a few
// long rows is spread over all CTAs like any other.
template <int DT, int OP>
__global__ void __launch_bounds__(256) k_reduce_box(const void *__restrict__ x, int64_t n_mid, int64_t n_inner,
                                                    int64_t s_outer, int64_t s_mid, int64_t n_seg,
                                                    int64_t items, double ident, double *partials,
                                                    unsigned *counter, double *result)
{
    __shared__ double wsum[8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t per = (items + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per;
    const int64_t i1 = i0 + per < items ? i0 + per : items;
    double acc = ident;
    for (int64_t it = i0 + warp; it < i1; it += nw) {
        const int64_t r = it / n_seg, sg = it - r * n_seg;
        const int64_t o = r / n_mid, m = r - o * n_mid;
        const int64_t c0 = sg * NOALLOC_SEG;
        const int64_t c1 = c0 + NOALLOC_SEG < n_inner ? c0 + NOALLOC_SEG : n_inner;
        const int64_t base = o * s_outer + m * s_mid;
        int64_t c = c0 + lane;
        for (; c + 96 < c1; c += 128) {
            const double v0 = ld<DT>(x, base + c), v1 = ld<DT>(x, base + c + 32);
            const double v2 = ld<DT>(x, base + c + 64), v3 = ld<DT>(x, base + c + 96);
            acc = fold<OP>(fold<OP>(fold<OP>(fold<OP>(acc, v0), v1), v2), v3);
        }
        for (; c < c1; c += 32) acc = fold<OP>(acc, ld<DT>(x, base + c));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = fold<OP>(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    if (lane == 0) wsum[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = wsum[0];
        for (int w = 1; w < nw; w++) b = fold<OP>(b, wsum[w]);
        partials[blockIdx.x] = b;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double *vp = partials;
        double s = vp[0];
        for (unsigned b = 1; b < gridDim.x; b++) s = fold<OP>(s, vp[b]);
        *result = s;
        *counter = 0u;
    }
}

template <int DT>
void launch_box(int op, int nblocks, cudaStream_t s, const void *x, int64_t n_mid, int64_t n_inner,
                int64_t s_outer, int64_t s_mid, int64_t n_seg, int64_t items, double *partials,
                unsigned *counter, double *result)
{
    const double inf = __builtin_inf();
    switch (op) {
    case 0: k_reduce_box<DT, 0><<<nblocks, 256, 0, s>>>(x, n_mid, n_inner, s_outer, s_mid, n_seg, items, 0.0, partials, counter, result); break;
    case 1: k_reduce_box<DT, 1><<<nblocks, 256, 0, s>>>(x, n_mid, n_inner, s_outer, s_mid, n_seg, items, 1.0, partials, counter, result); break;
    case 2: k_reduce_box<DT, 2><<<nblocks, 256, 0, s>>>(x, n_mid, n_inner, s_outer, s_mid, n_seg, items, -inf, partials, counter, result); break;
    default: k_reduce_box<DT, 3><<<nblocks, 256, 0, s>>>(x, n_mid, n_inner, s_outer, s_mid, n_seg, items, inf, partials, counter, result); break;
    }
}

}  // namespace

extern "C" int HDArrayReduceBufferNoAlloc(const void *x, const char *type, int dim, const int64_t *extent,
                                          const int64_t *strides, REDUCE_OP op, double *result,
                                          void *stream)
{
    if (!x || !type || !extent || !strides || !result || dim < 1 || dim > 3) return HDARRAY_ERR_INVAL;
    if ((int)op < 0 || (int)op > 3) return HDARRAY_ERR_INVAL;
    int dt;
    if (!strcmp(type, "double")) dt = hda::DT_F64;
    else if (!strcmp(type, "float")) dt = hda::DT_F32;
    else if (!strcmp(type, "bf16") || !strcmp(type, "bfloat16")) dt = hda::DT_BF16;
    else return HDARRAY_ERR_INVAL;
    if (strides[dim - 1] != 1) return HDARRAY_ERR_INVAL;  // the innermost dimension is contiguous
    int64_t n[3] = {1, 1, 1}, st[3] = {0, 0, 1};
    int64_t elems = 1;
    for (int d = 0; d < dim; d++) {
        if (extent[d] < 0) return HDARRAY_ERR_INVAL;
        n[3 - dim + d] = extent[d];
        st[3 - dim + d] = strides[d];
        if (extent[d] > 0 && elems > NOALLOC_MAX_ELEMS / extent[d]) return HDARRAY_ERR_RANGE;
        elems *= extent[d];
    }
    if (elems > NOALLOC_MAX_ELEMS) return HDARRAY_ERR_RANGE;  // beyond the per-call limit
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return HDARRAY_ERR_CUDA;
    }
    if (!g_scratch_addr[dev]) {  // set-up, once per device, with that device current
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HDARRAY_ERR_CUDA;
        }
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *partials = (double *)g_scratch_addr[dev];
    unsigned *counter = (unsigned *)(g_scratch_addr[dev] + NOALLOC_COUNTER_OFFSET);
    // work items: every row split into n_seg segments; an empty box has no items and one CTA
    // writes the operator's identity
    const int64_t n_seg = (n[2] + NOALLOC_SEG - 1) / NOALLOC_SEG;
    const int64_t items = elems == 0 ? 0 : n[0] * n[1] * n_seg;
    int64_t nb = (elems + 65535) / 65536;
    if (nb > NOALLOC_MAX_PARTIALS) nb = NOALLOC_MAX_PARTIALS;
    if (nb > items) nb = items;
    if (nb < 1) nb = 1;
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return HDARRAY_ERR_CUDA;
    }
    switch (dt) {
    case hda::DT_F64: launch_box<hda::DT_F64>((int)op, (int)nb, s, x, n[1], n[2], st[0], st[1], n_seg > 0 ? n_seg : 1, items, partials, counter, result); break;
    case hda::DT_F32: launch_box<hda::DT_F32>((int)op, (int)nb, s, x, n[1], n[2], st[0], st[1], n_seg > 0 ? n_seg : 1, items, partials, counter, result); break;
    default: launch_box<hda::DT_BF16>((int)op, (int)nb, s, x, n[1], n[2], st[0], st[1], n_seg > 0 ? n_seg : 1, items, partials, counter, result); break;
    }
    if (cudaGetLastError() != cudaSuccess) return HDARRAY_ERR_CUDA;
    return HDARRAY_OK;
}
