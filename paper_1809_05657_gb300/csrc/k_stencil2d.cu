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
#include "stencil_common.cuh"

namespace hda {

// One output row of a tile: up / mid / dn are the rows above, at and below.
template <int DT>
__device__ __forceinline__ void jacobi_row(const Row<DT> &up, const Row<DT> &mid, const Row<DT> &dn,
                                           typename Elem<DT>::E *yrow, int x, int c0, int c1, bool full,
                                           bool act, int lane)
{
    using EL = Elem<DT>;
    using A = typename EL::A;
    constexpr int VEC = EL::VEC;
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
    if (full) {
        *reinterpret_cast<typename EL::V *>(yrow) = EL::pack(out);
    } else if (act) {
#pragma unroll
        for (int k = 0; k < VEC; k++)
            if (x + k >= c0 && x + k < c1) EL::store1(yrow + k, out[k]);
    }
}

// NR rows live in a register ring: the row above, the row itself and NR - 2 rows ahead.  The march
// is unrolled by NR so that every ring slot is a fixed register set (no moves between steps):
// at unrolled step u of a group starting at output row r, slot u holds row r + u - 1, slot
// (u+1) % NR row r + u and slot (u+2) % NR row r + u + 1; after the step slot u is refilled with
// row r + u - 1 + NR.
template <int DT, int NR>
__global__ void __launch_bounds__(256) k_jacobi2d(const StenPart2D *__restrict__ parts,
                                                  const StenTile2D *__restrict__ tiles, int ntiles,
                                                  const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    constexpr int VEC = EL::VEC;
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= ntiles) return;  // warp-uniform
    const StenTile2D t = tiles[wid];
    const StenPart2D P = parts[t.part];

    receive_segments<E>(segs, t.seg0, t.nseg, lane);

    const int x = t.cb + lane * VEC;
    const bool act = (x < t.c1 + 1) && (x + VEC > t.c0 - 1);
    const bool needL = (t.cb >= t.c0) && (t.cb < t.c1);
    const bool needR = (t.cb + 32 * VEC - 1 >= t.c0) && (t.cb + 32 * VEC - 1 < t.c1);
    const bool full = (x >= t.c0) && (x + VEC <= t.c1);
    const int64_t xs = P.xs, ys = P.ys;
    const E *xp = reinterpret_cast<const E *>(P.x) + (int64_t)(t.r0 - 1 - P.xlo0) * xs + (x - P.xlo1);
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.r0 - P.ylo0) * ys + (x - P.ylo1);

    Row<DT> ring[NR];
#pragma unroll
    for (int k = 0; k < NR; k++) {
        if (t.r0 - 1 + k <= t.r1) load_row<DT>(ring[k], xp, 0, act, needL, needR, lane);
        xp += xs;
    }
    int r = t.r0;
    for (; r + NR <= t.r1; r += NR) {
#pragma unroll
        for (int u = 0; u < NR; u++) {
            jacobi_row<DT>(ring[u], ring[(u + 1) % NR], ring[(u + 2) % NR], yp, x, t.c0, t.c1, full, act, lane);
            yp += ys;
            if (r + u - 1 + NR <= t.r1) load_row<DT>(ring[u], xp, 0, act, needL, needR, lane);
            xp += xs;
        }
    }
#pragma unroll
    for (int u = 0; u < NR; u++) {
        if (r + u < t.r1) {
            jacobi_row<DT>(ring[u], ring[(u + 1) % NR], ring[(u + 2) % NR], yp, x, t.c0, t.c1, full, act, lane);
            yp += ys;
            if (r + u - 1 + NR <= t.r1) load_row<DT>(ring[u], xp, 0, act, needL, needR, lane);
            xp += xs;
        }
    }
}

// ------------------------------------------------------------------------------------------
// The same tile with the prefetched rows in shared memory instead of registers: every lane
// issues asynchronous 16-byte copies (cp.async) of its chunk of the rows ahead into a ring of NS
// stages owned by its warp, so the bytes in flight per SM are bounded by shared memory, not by
// registers.  Each lane reads back only what it copied itself (plus the band edges copied by lanes
// 0 and 31), so no synchronisation beyond cp.async.wait_group is needed; horizontal neighbours
// still come by shuffle.  Stage layout per warp: NS x (32 chunks + 2 edge slots) x 16 bytes.
// ------------------------------------------------------------------------------------------
template <int DT, int NS>
__global__ void __launch_bounds__(256) k_jacobi2d_async(const StenPart2D *__restrict__ parts,
                                                        const StenTile2D *__restrict__ tiles,
                                                        int ntiles, const Seg *__restrict__ segs)
{
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    constexpr int VEC = EL::VEC;
    constexpr int SLOTS = 34;  // 32 chunks + left edge + right edge
    extern __shared__ uint4 smem[];
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wid >= ntiles) return;  // warp-uniform
    uint4 *ring = smem + (threadIdx.x >> 5) * NS * SLOTS;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
    const StenTile2D t = tiles[wid];
    const StenPart2D P = parts[t.part];

    receive_segments<E>(segs, t.seg0, t.nseg, lane);

    const int x = t.cb + lane * VEC;
    const bool act = (x < t.c1 + 1) && (x + VEC > t.c0 - 1);
    const bool needL = (t.cb >= t.c0) && (t.cb < t.c1);
    const bool needR = (t.cb + 32 * VEC - 1 >= t.c0) && (t.cb + 32 * VEC - 1 < t.c1);
    const bool full = (x >= t.c0) && (x + VEC <= t.c1);
    const bool doL = lane == 0 && needL, doR = lane == 31 && needR;
    const int64_t xs = P.xs, ys = P.ys;
    const E *xp = reinterpret_cast<const E *>(P.x) + (int64_t)(t.r0 - 1 - P.xlo0) * xs + (x - P.xlo1);
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.r0 - P.ylo0) * ys + (x - P.ylo1);

    // prologue: rows r0-1 .. r0-2+NS into stages 0 .. NS-1
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (t.r0 - 1 + s <= t.r1) {
            const uint32_t sa = ring_s + (uint32_t)(s * SLOTS) * 16u;
            if (act) cpa16(sa + lane * 16u, xp);
            if (doL) edge_copy<DT>(sa + 32u * 16u, xp - 1, true);
            if (doR) edge_copy<DT>(sa + 33u * 16u, xp + VEC, false);
        }
        cpa_commit();
        xp += xs;
    }
    for (int r = t.r0; r < t.r1; r++) {
        const int k = r - t.r0;
        cpa_wait<NS - 3>();  // rows up to r + 1 have landed
        const uint4 *su = ring + (k % NS) * SLOTS, *sm = ring + ((k + 1) % NS) * SLOTS,
                    *sd = ring + ((k + 2) % NS) * SLOTS;
        Row<DT> up, mid, dn;
        if (act) {
            EL::unpack(*reinterpret_cast<const typename EL::V *>(su + lane), up.v);
            EL::unpack(*reinterpret_cast<const typename EL::V *>(sm + lane), mid.v);
            EL::unpack(*reinterpret_cast<const typename EL::V *>(sd + lane), dn.v);
        }
        if (doL) mid.l = edge_read<DT>(sm + 32, true);
        if (doR) mid.r = edge_read<DT>(sm + 33, false);
        jacobi_row<DT>(up, mid, dn, yp, x, t.c0, t.c1, full, act, lane);
        yp += ys;
        // the row above is done with: refill its stage with row r - 1 + NS
        if (r - 1 + NS <= t.r1) {
            const uint32_t sa = ring_s + (uint32_t)((k % NS) * SLOTS) * 16u;
            if (act) cpa16(sa + lane * 16u, xp);
            if (doL) edge_copy<DT>(sa + 32u * 16u, xp - 1, true);
            if (doR) edge_copy<DT>(sa + 33u * 16u, xp + VEC, false);
        }
        cpa_commit();
        xp += xs;
    }
    cpa_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Packed-stream variant for partitions of any width: one CTA of 256 threads per tile of a column
// band of nch 16-byte chunks (nch <= 32) and ns * sl rows, cut into ns streams of sl consecutive
// rows (ns * nch <= 256, one chunk per thread), all streams marching down their rows in step.  A
// narrow band (the column partitions of a small instance) so keeps every lane busy with several
// row streams instead of idling most of a warp.  Entry e of a stream is its row r_s - 1 + e
// (e = 0 .. len_s + 1; r_s its first row); entry e of every stream -- nch chunks plus one halo chunk
// on each side, each halo chunk only where the band's output range ends on a chunk boundary -- goes
// into stage e % NS of a shared-memory ring by cp.async.  A step computes output rows r_s + k and
// r_s + k + 1 from entries k .. k+3 after refilling the stages of entries k-2, k-1 (free since the
// barrier of this step) with entries k+NS-2, k+NS-1.  A stage is stage_slots >= ns * (nch + 2)
// slots of 16 bytes, at most 512.
//
// OP selects the point operation on the 3 x 3 neighbourhood: OP_JACOBI, the Jacobi step above;
// OP_CONV, the 2-D convolution of Sec. 5 (eight neighbours and the centre) with the weights w[9]:
//   Y[i][j] = sum over a, b in 0..2 of w[3a + b] * X[i+a-1][j+b-1],
// accumulated in that row-major order, each product rounded (no fused multiply-add), in the
// arithmetic precision (binary32 for bfloat16 storage; weights rounded to it).
// ------------------------------------------------------------------------------------------
constexpr int OP_JACOBI = 0, OP_CONV = 1;

template <typename A>
__device__ __forceinline__ A mul_rn(A a, A b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename A>
__device__ __forceinline__ A add_rn(A a, A b);
template <>
__device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }

template <int DT, int NS, int OP>
__global__ void __launch_bounds__(256, 4) k_jacobi2d_cta(const StenPart2D *__restrict__ parts,
                                                        const StenTile2D *__restrict__ tiles, int stage_slots,
                                                        const Seg *__restrict__ segs, const double *__restrict__ wts)
{
    static_assert((NS & (NS - 1)) == 0 && NS >= 6, "ring depth: a power of two, at least 6");
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    using V = typename EL::V;
    constexpr int VEC = EL::VEC;
    extern __shared__ uint4 smem[];
    const int lane = threadIdx.x & 31;
    const StenTile2D t = tiles[blockIdx.x];
    const StenPart2D P = parts[t.part];
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(smem);
    A w[9];
#pragma unroll
    for (int k = 0; k < 9; k++) w[k] = OP == OP_CONV ? (A)wts[k] : A(0);

    receive_segments_cta<E, DT != DT_BF16>(segs, t.seg0, t.nseg);

    const int nch = t.nch, rw = nch + 2, G = t.ns, SL = t.sl;
    const int SS = G * rw;                        // 16-byte slots used per stage
    const bool needL = t.c0 == t.cb;              // c0 - 1 lies in the left halo chunk
    const bool needR = t.c1 == t.cb + nch * VEC;  // c1 lies in the right halo chunk

    // This thread's copy items: slots j and j + 256 of every entry, (stream, chunk) = divmod(j, rw),
    // each loaded while its stream has rows left (entries 0 .. len + 1).
    const int j0 = threadIdx.x, j1 = threadIdx.x + 256;
    const int s0 = j0 / rw, q0 = j0 - s0 * rw, s1 = j1 / rw, q1 = j1 - s1 * rw;
    const bool has0 = j0 < SS && (q0 > 0 || needL) && (q0 < rw - 1 || needR);
    const bool has1 = j1 < SS && (q1 > 0 || needL) && (q1 < rw - 1 || needR);
    const int last0 = min(SL, t.r1 - t.r0 - s0 * SL) + 1, last1 = min(SL, t.r1 - t.r0 - s1 * SL) + 1;
    const int64_t xs = P.xs;
    const E *xrow = reinterpret_cast<const E *>(P.x) + (t.cb - VEC - P.xlo1);  // column of slot 0, row 0
    const E *src0 = xrow + (int64_t)(t.r0 + s0 * SL - 1 - P.xlo0) * xs + q0 * VEC;
    const E *src1 = xrow + (int64_t)(t.r0 + s1 * SL - 1 - P.xlo0) * xs + q1 * VEC;
    const uint32_t stage_bytes = (uint32_t)stage_slots * 16u;
    int enext = 0;  // next entry to issue
    auto issue = [&]() {
        const uint32_t sb = ring_s + (uint32_t)(enext & (NS - 1)) * stage_bytes;
        if (has0 && enext <= last0) cpa16(sb + (uint32_t)j0 * 16u, src0);
        if (has1 && enext <= last1) cpa16(sb + (uint32_t)j1 * 16u, src1);
        src0 += xs;
        src1 += xs;
        enext++;
        cpa_commit();  // one group per entry
    };
#pragma unroll 1
    for (int k = 0; k < NS - 2; k++) issue();  // entries 0 .. NS-3

    // the chunk this thread computes: stream s, chunk c
    const int s = threadIdx.x / nch, c = threadIdx.x - s * nch;
    const int x = t.cb + c * VEC;
    const bool act = s < G;
    const int len = act ? min(SL, t.r1 - t.r0 - s * SL) : 0;  // output rows of this stream
    const bool full = x >= t.c0 && x + VEC <= t.c1;
    const int me = s * rw + c + 1;
    const bool shflL = c > 0 && lane > 0, shflR = c < nch - 1 && lane < 31;
    const bool haveL = c > 0 || needL, haveR = c < nch - 1 || needR;
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.r0 + s * SL - P.ylo0) * P.ys + (x - P.ylo1);

    auto ld = [&](int e, A (&v)[VEC]) {  // this thread's chunk of entry e
        if (act) EL::unpack(*reinterpret_cast<const V *>(smem + (e & (NS - 1)) * stage_slots + me), v);
    };
    // the elements left and right of this thread's chunk of entry e (v holds the chunk)
    auto ends = [&](int e, const A (&v)[VEC], A &left, A &right) {
        left = __shfl_up_sync(0xffffffffu, v[VEC - 1], 1);
        right = __shfl_down_sync(0xffffffffu, v[0], 1);
        const E *sr = reinterpret_cast<const E *>(smem + (e & (NS - 1)) * stage_slots + me);
        if (!shflL && act && haveL) left = EL::load1(sr - 1);
        if (!shflR && act && haveR) right = EL::load1(sr + VEC);
    };
    // one output row from the entries e-1, e, e+1 (rows above, centre, below); stored at out_p
    auto row = [&](int e, const A (&up)[VEC], const A (&cv)[VEC], const A (&dn)[VEC], E *out_p, bool store) {
        A out[VEC];
        A cl, cr;
        ends(e, cv, cl, cr);
        if constexpr (OP == OP_JACOBI) {
#pragma unroll
            for (int k = 0; k < VEC; k++) {
                const A wv = k > 0 ? cv[k - 1] : cl;
                const A ev = k < VEC - 1 ? cv[k + 1] : cr;
                A sum = wv + ev;
                sum = sum + up[k];
                sum = sum + dn[k];
                out[k] = sum * A(0.25);
            }
        } else {
            A ul, ur, dl, dr;
            ends(e - 1, up, ul, ur);
            ends(e + 1, dn, dl, dr);
#pragma unroll
            for (int k = 0; k < VEC; k++) {
                const A r0[3] = {k > 0 ? up[k - 1] : ul, up[k], k < VEC - 1 ? up[k + 1] : ur};
                const A r1[3] = {k > 0 ? cv[k - 1] : cl, cv[k], k < VEC - 1 ? cv[k + 1] : cr};
                const A r2[3] = {k > 0 ? dn[k - 1] : dl, dn[k], k < VEC - 1 ? dn[k + 1] : dr};
                A sum = mul_rn(w[0], r0[0]);
                sum = add_rn(sum, mul_rn(w[1], r0[1]));
                sum = add_rn(sum, mul_rn(w[2], r0[2]));
                sum = add_rn(sum, mul_rn(w[3], r1[0]));
                sum = add_rn(sum, mul_rn(w[4], r1[1]));
                sum = add_rn(sum, mul_rn(w[5], r1[2]));
                sum = add_rn(sum, mul_rn(w[6], r2[0]));
                sum = add_rn(sum, mul_rn(w[7], r2[1]));
                sum = add_rn(sum, mul_rn(w[8], r2[2]));
                out[k] = sum;
            }
        }
        if (store) {
            if (full) {
                *reinterpret_cast<V *>(out_p) = EL::pack(out);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (x + k >= t.c0 && x + k < t.c1) EL::store1(out_p + k, out[k]);
            }
        }
    };

    // A step computes output rows r_s + k and r_s + k + 1 from entries k .. k+3.  Entries k and
    // k + 1 are the previous step's k + 2 and k + 3, still unpacked in registers, so every entry
    // is read from shared memory and unpacked once; the loop body is two steps with the four row
    // register sets exchanging roles, so no values move between registers.
    auto step = [&](int k, A (&e0)[VEC], A (&e1)[VEC], A (&e2)[VEC], A (&e3)[VEC], bool first) {
        cpa_wait<NS - 6>();  // entries up to k + 3 have landed (this thread's copies)
        __syncthreads();     // ... and every other thread's; the stages of k-2 and k-1 are free
        issue();             // entry k + NS - 2
        issue();             // entry k + NS - 1
        if (first) {
            ld(k, e0);
            ld(k + 1, e1);
        }
        ld(k + 2, e2);
        row(k + 1, e0, e1, e2, yp, k < len);  // output row r_s + k
        if (k + 1 < SL) {                     // output row r_s + k + 1
            ld(k + 3, e3);
            row(k + 2, e1, e2, e3, yp + P.ys, k + 1 < len);
        }
        yp += 2 * P.ys;
    };
    A ra[VEC], rb[VEC], rc[VEC], rd[VEC];
    step(0, ra, rb, rc, rd, true);
    for (int k = 2; k < SL; k += 4) {
        step(k, rc, rd, ra, rb, false);
        if (k + 2 < SL) step(k + 2, ra, rb, rc, rd, false);
    }
    cpa_wait<0>();
}

cudaError_t launch_stencil2d_cta(int op, int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                 const Seg *segs, const double *weights, size_t smem, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    constexpr int NS = JACOBI2D_STAGES;
    const int slots = (int)(smem / ((size_t)NS * 16));
    if (slots < 1 || slots > 512 || smem != (size_t)NS * slots * 16) return cudaErrorInvalidValue;
    const int which = dtype == DT_F64 ? 0 : dtype == DT_F32 ? 1 : dtype == DT_BF16 ? 2 : -1;
    if (which < 0 || (op != OP_JACOBI && op != OP_CONV) || (op == OP_CONV && !weights)) return cudaErrorInvalidValue;
    using KFn = void (*)(const StenPart2D *, const StenTile2D *, int, const Seg *, const double *);
    const KFn fns[2][3] = {{k_jacobi2d_cta<DT_F64, NS, OP_JACOBI>, k_jacobi2d_cta<DT_F32, NS, OP_JACOBI>,
                            k_jacobi2d_cta<DT_BF16, NS, OP_JACOBI>},
                           {k_jacobi2d_cta<DT_F64, NS, OP_CONV>, k_jacobi2d_cta<DT_F32, NS, OP_CONV>,
                            k_jacobi2d_cta<DT_BF16, NS, OP_CONV>}};
    static bool attr[2][3] = {};
    if (!attr[op][which]) {
        cudaError_t e = cudaFuncSetAttribute(fns[op][which], cudaFuncAttributeMaxDynamicSharedMemorySize, NS * 512 * 16);
        if (e != cudaSuccess) return e;
        attr[op][which] = true;
    }
    fns[op][which]<<<ntiles, 256, smem, s>>>(parts, tiles, slots, segs, weights);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// The Jacobi step (OP_JACOBI) or the 3 x 3 convolution (OP_CONV, the order and rounding of the
// packed-stream form above) with its rows staged by the tensor memory accelerator.  A tile is a column band
// of nch 16-byte chunks by rows r0 .. r1 - 1 of one device, cut into stages of SR = ns * M output
// rows.  Stage j is one box of the part's 2-D tensor map: the SR + 2 buffer rows
// r0 - 1 + j * SR .. r0 + (j + 1) * SR (both halo rows included) by rwb chunks (the band with one
// halo chunk on each side), brought by a single bulk tensor copy (cp.async.bulk.tensor.2d) that
// thread 0 issues into a ring of NS stages and that completes a transaction-count mbarrier.
// Thread (g, c) computes chunk c of the M consecutive output rows g * M .. g * M + M - 1 of every
// stage: it reads its M + 2 staged rows from shared memory once each, the three-row window sliding
// down in registers, and the copies cost the computing threads no instructions.  Horizontal
// neighbours come by shuffle, or from the staged halo chunks, which every box holds (coordinates
// outside the buffer read zeros, never used by an output); the convolution takes them for every
// staged row once per stage, the Jacobi step for the centre row of each output row.  The tile
// copies its receive segments -- the parts of the sections its device receives in this call
// (Eq. 1-2) that only this tile reads -- from the senders' buffers into its own, and every thread
// fences those generic stores to the async proxy.  Without RX, or with more than rx_cap received
// elements, it does so before its first copy.  With RX it issues the ring's first NS copies
// first, so that they fly during the receive, and keeps each received value with its place in the
// tile's staged window in shared memory.  When one of those stages has landed, the threads write
// the values into it before anyone reads it.  Later stages are issued after the fence and read
// the values from the buffer.  Waits are bounded: after spin_limit polls a wait gives up, the tile
// stops, thread 0 waits (with a fixed limit) for the copies it issued and the error word is set.
// ------------------------------------------------------------------------------------------

// The receive of a tile with RX: this thread's elements e = threadIdx.x + q * blockDim.x (q < 4)
// of its segments, flattened in order, loaded together, then stored into the own buffer xb (row
// stride xs elements) and kept at side_v[e] with side_p[e] = (row << 9) | column: the element's
// place relative to the staged window's first row yc and the box's first column xc (buffer
// coordinates), or -1 outside the window (never patched).
template <typename E>
__device__ __forceinline__ void receive_keep(const Seg *__restrict__ segs, int seg0, int nseg, const E *xb, int64_t xs,
                                             int64_t yc, int64_t xc, E *side_v, int32_t *side_p)
{
    E v[4];
    E *dp[4];
    int32_t pp[4];
    int u = 0, e = threadIdx.x, i0 = 0;
    for (int s = 0; s < nseg && u < 4; s++) {
        const Seg g = segs[seg0 + s];
        const int total = g.n * g.m;
        while (u < 4 && e < i0 + total) {
            const int i = e - i0, o = i / g.n, k = i - o * g.n;
            const E *sp = reinterpret_cast<const E *>(g.src) + (o * g.sso + k * g.ss);
            E *dq = reinterpret_cast<E *>(g.dst) + (o * g.dso + k * g.ds);
            const int64_t off = dq - xb;
            const int64_t r = (off >= 0 && off < INT32_MAX && xs < INT32_MAX) ? (int64_t)((uint32_t)off / (uint32_t)xs)
                                                                            : off / xs;
            const int64_t tr = r - yc, tc = off - r * xs - xc;
            const int32_t p = (tr >= 0 && tr < (1 << 21) && tc >= 0 && tc < 512) ? (int32_t)((tr << 9) | tc) : -1;
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (q == u) {
                    v[q] = *sp;
                    dp[q] = dq;
                    pp[q] = p;
                }
            u++;
            e += blockDim.x;
        }
        i0 += total;
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (q < u) {
            *dp[q] = v[q];
            side_v[threadIdx.x + q * blockDim.x] = v[q];
            side_p[threadIdx.x + q * blockDim.x] = pp[q];
        }
}

template <int DT, int NS, int M, int OP, bool RX>
__global__ void __launch_bounds__(256, 3) k_jacobi2d_tma(const StenPart2D *__restrict__ parts,
                                                         const StenTile2D *__restrict__ tiles,
                                                         const Seg *__restrict__ segs,
                                                         const uint8_t *__restrict__ tmaps, const double *__restrict__ wts,
                                                         unsigned *err, unsigned spin_limit, int ring_bytes, int rx_cap)
{
    static_assert((NS & (NS - 1)) == 0 && NS >= 2, "ring depth: a power of two");
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    using V = typename EL::V;
    constexpr int VEC = EL::VEC;
    extern __shared__ uint4 smem_dyn[];
    __shared__ __align__(8) uint64_t full[NS];
    const int lane = threadIdx.x & 31;
    const StenTile2D t = tiles[blockIdx.x];
    const StenPart2D P = parts[t.part];
    A w[9];
#pragma unroll
    for (int k = 0; k < 9; k++) w[k] = OP == OP_CONV ? (A)wts[k] : A(0);
    // the ring starts on a 128-byte boundary (the launch adds 128 bytes of slack)
    const uint32_t ring_s = (smem_addr(smem_dyn) + 127u) & ~127u;
    const char *ring = reinterpret_cast<const char *>(smem_dyn) + (ring_s - smem_addr(smem_dyn));

    // RX: the received values and their places, after the ring
    E *side_v = reinterpret_cast<E *>(reinterpret_cast<char *>(smem_dyn) + ring_bytes);
    int32_t *side_p = reinterpret_cast<int32_t *>(side_v + rx_cap);
    int ntot = 0;  // RX: received elements of the tile
    if (RX)
        for (int s = 0; s < t.nseg; s++) ntot += segs[t.seg0 + s].n * segs[t.seg0 + s].m;
    const bool late = RX && t.nseg > 0 && ntot <= rx_cap;
    if (t.nseg > 0 && !late) receive_flat_vec<E>(segs, t.seg0, t.nseg, threadIdx.x, blockDim.x);
    asm volatile("fence.proxy.async.global;" ::: "memory");  // the receive's stores, before bulk copies read them
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int nch = t.nch, G = t.ns, rw = P.rwb;  // chunks computed, row groups, staged row width
    const int SR = G * M;                          // output rows per stage
    const int S = (t.r1 - t.r0 + SR - 1) / SR;     // stages of the tile
    const uint32_t box_bytes = (uint32_t)(SR + 2) * (uint32_t)rw * 16u;
    const uint32_t stage_bytes = (box_bytes + 127u) & ~127u;
    const uint8_t *tmap = tmaps + (size_t)t.part * 128;
    const int xc = (int)(t.cb - VEC - P.xlo1), yc = (int)(t.r0 - 1 - P.xlo0);
    int issued = 0;  // thread 0: stages issued so far
    auto issue = [&](int j) {
        if (j >= S) return;
        const uint32_t bar = smem_addr(&full[j & (NS - 1)]);
        const uint32_t dst = ring_s + (uint32_t)(j & (NS - 1)) * stage_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(box_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
            "l"(tmap), "r"(xc), "r"(yc + j * SR), "r"(bar)
            : "memory");
        issued = j + 1;
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < NS; j++) issue(j);
    if (late) {
        // stages NS and later are issued after the first barrier of the loop, so after this fence
        receive_keep<E>(segs, t.seg0, t.nseg, reinterpret_cast<const E *>(P.x), P.xs, yc, xc, side_v, side_p);
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }

    // this thread: row group gi (output rows gi * M .. of every stage), chunk c
    const int gi = threadIdx.x / nch, c = threadIdx.x - gi * nch;
    const bool act = gi < G;
    const int x = t.cb + c * VEC;
    const bool full_chunk = x >= t.c0 && x + VEC <= t.c1;
    const bool shflL = c > 0 && lane > 0, shflR = c < nch - 1 && lane < 31;
    // slot of the thread's chunk in its first staged row; the idle threads past the last row group
    // read the first rows (valid shared memory) and store nothing, so every thread runs the same
    // instructions (no selects around the loads and unpacking)
    const int me = (act ? gi * M * rw : 0) + c + 1;
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.r0 + gi * M - P.ylo0) * P.ys + (x - P.ylo1);

    bool failed = false;
    for (int j = 0; j < S; j++) {
        const bool ok = mbar_wait_bounded(smem_addr(&full[j & (NS - 1)]), (uint32_t)((j / NS) & 1), spin_limit);
        // every thread is done with stage j - 1; a failed wait anywhere stops every thread
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (late && j < NS) {
            // this stage was copied before the receive's stores: the received values go in now,
            // ordered before any later bulk copy into the same slot
            char *st = const_cast<char *>(ring) + (size_t)(j & (NS - 1)) * stage_bytes;
            for (int e = threadIdx.x; e < ntot; e += blockDim.x) {
                const int32_t p = side_p[e];
                const int ir = (p >> 9) - j * SR, ic = p & 511;
                if (p >= 0 && ir >= 0 && ir < SR + 2 && ic < rw * VEC)
                    *reinterpret_cast<E *>(st + (size_t)ir * rw * 16 + (size_t)ic * sizeof(E)) = side_v[e];
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
        }
        if (threadIdx.x == 0 && j > 0) issue(j - 1 + NS);
        const uint4 *sp = reinterpret_cast<const uint4 *>(ring + (size_t)(j & (NS - 1)) * stage_bytes) + me;
        const int rbase = t.r0 + j * SR + gi * M;  // the thread's first output row in this stage
        A rows[M + 2][VEC];
#pragma unroll
        for (int q = 0; q < M + 2; q++) EL::unpack(*reinterpret_cast<const V *>(sp + q * rw), rows[q]);
        // the elements left and right of the thread's chunk in staged row q: by shuffle, or from the
        // staged neighbouring chunk (every box holds the halo chunks)
        auto ends = [&](int q, A &left, A &right) {
            left = __shfl_up_sync(0xffffffffu, rows[q][VEC - 1], 1);
            right = __shfl_down_sync(0xffffffffu, rows[q][0], 1);
            const E *crow = reinterpret_cast<const E *>(sp + q * rw);
            if (!shflL) left = EL::load1(crow - 1);
            if (!shflR) right = EL::load1(crow + VEC);
        };
        A lft[M + 2], rgt[M + 2];  // the convolution's: every staged row's, once
        if constexpr (OP == OP_CONV) {
#pragma unroll
            for (int q = 0; q < M + 2; q++) ends(q, lft[q], rgt[q]);
        }
#pragma unroll
        for (int u = 0; u < M; u++) {
            const A(&up)[VEC] = rows[u];
            const A(&cv)[VEC] = rows[u + 1];
            const A(&dn)[VEC] = rows[u + 2];
            A out[VEC];
            if constexpr (OP == OP_JACOBI) {
                A left, right;
                ends(u + 1, left, right);
#pragma unroll
                for (int k = 0; k < VEC; k++) {
                    const A wv = k > 0 ? cv[k - 1] : left;
                    const A ev = k < VEC - 1 ? cv[k + 1] : right;
                    A sum = wv + ev;
                    sum = sum + up[k];
                    sum = sum + dn[k];
                    out[k] = sum * A(0.25);
                }
            } else {
#pragma unroll
                for (int k = 0; k < VEC; k++) {
                    const A r0[3] = {k > 0 ? up[k - 1] : lft[u], up[k], k < VEC - 1 ? up[k + 1] : rgt[u]};
                    const A r1[3] = {k > 0 ? cv[k - 1] : lft[u + 1], cv[k], k < VEC - 1 ? cv[k + 1] : rgt[u + 1]};
                    const A r2[3] = {k > 0 ? dn[k - 1] : lft[u + 2], dn[k], k < VEC - 1 ? dn[k + 1] : rgt[u + 2]};
                    A sum = mul_rn(w[0], r0[0]);
                    sum = add_rn(sum, mul_rn(w[1], r0[1]));
                    sum = add_rn(sum, mul_rn(w[2], r0[2]));
                    sum = add_rn(sum, mul_rn(w[3], r1[0]));
                    sum = add_rn(sum, mul_rn(w[4], r1[1]));
                    sum = add_rn(sum, mul_rn(w[5], r1[2]));
                    sum = add_rn(sum, mul_rn(w[6], r2[0]));
                    sum = add_rn(sum, mul_rn(w[7], r2[1]));
                    sum = add_rn(sum, mul_rn(w[8], r2[2]));
                    out[k] = sum;
                }
            }
            if (act && rbase + u < t.r1) {
                E *op = yp + (int64_t)(j * SR + u) * P.ys;
                if (full_chunk) {
                    *reinterpret_cast<V *>(op) = EL::pack(out);
                } else {
#pragma unroll
                    for (int k = 0; k < VEC; k++)
                        if (x + k >= t.c0 && x + k < t.c1) EL::store1(op + k, out[k]);
                }
            }
        }
    }
    if (failed && threadIdx.x == 0) {
        // the copies issued land before the CTA's shared memory is released: the last one of each
        // stage completes that stage's latest phase
        for (int j = issued - 1; j >= 0 && j >= issued - NS; j--)
            mbar_wait_bounded(smem_addr(&full[j & (NS - 1)]), (uint32_t)((j / NS) & 1), TMA_DRAIN_LIMIT);
        if (err) atomicOr(err, 1u);
    }
}

cudaError_t launch_jacobi2d_tma(int op, int dtype, const StenPart2D *parts, const StenTile2D *tiles, int ntiles,
                                const Seg *segs, size_t smem, cudaStream_t s, const void *tmaps, const double *weights,
                                unsigned *err, unsigned spin_limit, int rx_cap)
{
    if (ntiles <= 0) return cudaSuccess;
    constexpr int NS = JACOBI2D_TMA_STAGES, M = JACOBI2D_TMA_ROWS;
    const int which = dtype == DT_F64 ? 0 : dtype == DT_F32 ? 1 : dtype == DT_BF16 ? 2 : -1;
    if (which < 0 || (op != OP_JACOBI && op != OP_CONV) || (op == OP_CONV && !weights)) return cudaErrorInvalidValue;
    if (rx_cap < 0 || rx_cap > JACOBI2D_TMA_RX_MAX || rx_cap % JACOBI2D_TMA_THREADS != 0) return cudaErrorInvalidValue;
    const size_t esize = which == 0 ? 8 : which == 1 ? 4 : 2;
    // the ring's bytes are a multiple of 16 so that the received values after it stay aligned
    const size_t total = smem + (size_t)rx_cap * (esize + 4);
    if (!tmaps || smem < 128 || smem % 16 != 0 || total > (size_t)JACOBI2D_TMA_SMEM_MAX) return cudaErrorInvalidValue;
    using KFn = void (*)(const StenPart2D *, const StenTile2D *, const Seg *, const uint8_t *, const double *, unsigned *,
                         unsigned, int, int);
    const KFn fns[2][2][3] = {
        {{k_jacobi2d_tma<DT_F64, NS, M, OP_JACOBI, false>, k_jacobi2d_tma<DT_F32, NS, M, OP_JACOBI, false>,
          k_jacobi2d_tma<DT_BF16, NS, M, OP_JACOBI, false>},
         {k_jacobi2d_tma<DT_F64, NS, M, OP_CONV, false>, k_jacobi2d_tma<DT_F32, NS, M, OP_CONV, false>,
          k_jacobi2d_tma<DT_BF16, NS, M, OP_CONV, false>}},
        {{k_jacobi2d_tma<DT_F64, NS, M, OP_JACOBI, true>, k_jacobi2d_tma<DT_F32, NS, M, OP_JACOBI, true>,
          k_jacobi2d_tma<DT_BF16, NS, M, OP_JACOBI, true>},
         {k_jacobi2d_tma<DT_F64, NS, M, OP_CONV, true>, k_jacobi2d_tma<DT_F32, NS, M, OP_CONV, true>,
          k_jacobi2d_tma<DT_BF16, NS, M, OP_CONV, true>}}};
    const int rx = rx_cap > 0 ? 1 : 0;
    static bool attr[2][2][3] = {};
    if (!attr[rx][op][which]) {
        cudaError_t e = cudaFuncSetAttribute(fns[rx][op][which], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             JACOBI2D_TMA_SMEM_MAX);
        if (e != cudaSuccess) return e;
        attr[rx][op][which] = true;
    }
    fns[rx][op][which]<<<ntiles, 256, total, s>>>(parts, tiles, segs, reinterpret_cast<const uint8_t *>(tmaps), weights,
                                                  err, spin_limit, (int)smem, rx_cap);
    return cudaGetLastError();
}

cudaError_t launch_jacobi2d(int dtype, const StenPart2D *parts, const StenTile2D *tiles,
                            int ntiles, const Seg *segs, int warps_per_cta, int variant, size_t smem,
                            cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (variant == 3) return launch_stencil2d_cta(OP_JACOBI, dtype, parts, tiles, ntiles, segs, nullptr, smem, s);
    if (warps_per_cta < 1 || warps_per_cta > 8) warps_per_cta = 4;
    const int grid = (ntiles + warps_per_cta - 1) / warps_per_cta;
    const int block = 32 * warps_per_cta;
    if (variant == 1) {
        constexpr int NS = 8;
        const size_t sm = (size_t)warps_per_cta * NS * 34 * 16;
        switch (dtype) {
        case DT_F64: k_jacobi2d_async<DT_F64, NS><<<grid, block, sm, s>>>(parts, tiles, ntiles, segs); break;
        case DT_F32: k_jacobi2d_async<DT_F32, NS><<<grid, block, sm, s>>>(parts, tiles, ntiles, segs); break;
        case DT_BF16: k_jacobi2d_async<DT_BF16, NS><<<grid, block, sm, s>>>(parts, tiles, ntiles, segs); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (dtype) {
    case DT_F64: k_jacobi2d<DT_F64, 6><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_F32: k_jacobi2d<DT_F32, 6><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    case DT_BF16: k_jacobi2d<DT_BF16, 5><<<grid, block, 0, s>>>(parts, tiles, ntiles, segs); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hda
