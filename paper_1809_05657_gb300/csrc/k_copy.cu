// k_copy.cu -- section copy between logical-device buffers: the message of Eq. 1-2 moved on the
// GPU.  The paper reads each section out with clEnqueueReadBufferRect, sends it over MPI and
// writes it with clEnqueueWriteBufferRect (Sec. 3.1, HDArrayApplyKernel); here source and
// destination are device buffers of the same GPU and one kernel moves every section of a call.
//
// Each CTA copies one task (a slice of rows of one box) with the widest access the task's
// alignment allows (16-byte vectors for buffers whose rows start on 16-byte boundaries).  Every
// thread keeps four loads in flight before it stores them: rows of 128 chunks or more go a warp
// per row, lanes on consecutive chunks; shorter rows -- the faces of a partition, down to the
// one-element rows of 2-D column faces and 3-D x-faces -- are flattened into (row, chunk) items,
// consecutive threads on consecutive items.
#include "kernels.h"

namespace hda {

template <int V>
struct VecOf;
template <>
struct VecOf<16> {
    using T = uint4;
};
template <>
struct VecOf<8> {
    using T = uint2;
};
template <>
struct VecOf<4> {
    using T = uint32_t;
};
template <>
struct VecOf<2> {
    using T = uint16_t;
};

template <int V>
__device__ __forceinline__ void copy_task(const CopyTask &t)
{
    using T = typename VecOf<V>::T;
    constexpr int UNR = 4;
    const int nch = t.inner / V;
    const int nrows = t.row_end - t.row_begin;
    if (nch >= 32 * UNR) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int r = warp; r < nrows; r += nw) {
            const int row = t.row_begin + r;
            const int o = row / t.n_mid, m = row - o * t.n_mid;
            const T *s = reinterpret_cast<const T *>(t.src + o * t.s_outer + m * t.s_mid);
            T *d = reinterpret_cast<T *>(t.dst + o * t.d_outer + m * t.d_mid);
            for (int c0 = lane; c0 < nch; c0 += 32 * UNR) {
                T v[UNR];
#pragma unroll
                for (int u = 0; u < UNR; u++)
                    if (c0 + 32 * u < nch) v[u] = s[c0 + 32 * u];
#pragma unroll
                for (int u = 0; u < UNR; u++)
                    if (c0 + 32 * u < nch) d[c0 + 32 * u] = v[u];
            }
        }
        return;
    }
    const int total = nrows * nch;
    const int step = blockDim.x;
    for (int base = threadIdx.x; base < total; base += UNR * step) {
        T v[UNR];
        T *d[UNR];
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            d[u] = nullptr;
            const int i = base + u * step;
            if (i >= total) continue;
            const int r = i / nch, c = i - r * nch;
            const int row = t.row_begin + r;
            const int o = row / t.n_mid, m = row - o * t.n_mid;
            v[u] = reinterpret_cast<const T *>(t.src + o * t.s_outer + m * t.s_mid)[c];
            d[u] = reinterpret_cast<T *>(t.dst + o * t.d_outer + m * t.d_mid) + c;
        }
#pragma unroll
        for (int u = 0; u < UNR; u++)
            if (d[u]) *d[u] = v[u];
    }
}

__global__ void __launch_bounds__(256) k_section_copy(const CopyTask *__restrict__ tasks)
{
    const CopyTask t = tasks[blockIdx.x];
    switch (t.vec) {
    case 16: copy_task<16>(t); break;
    case 8: copy_task<8>(t); break;
    case 4: copy_task<4>(t); break;
    default: copy_task<2>(t); break;
    }
}

cudaError_t launch_copy(const CopyTask *tasks, int ntasks, cudaStream_t s)
{
    if (ntasks <= 0) return cudaSuccess;
    k_section_copy<<<ntasks, 256, 0, s>>>(tasks);
    return cudaGetLastError();
}

}  // namespace hda
