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
    load_row<DT, true>(zm, Xc + (int64_t)(t.z0 - 1 - zx) * zs, 0, act, false, false, lane);
    load_row<DT, true>(zc, Xc + (int64_t)(t.z0 - zx) * zs, 0, act, needL, needR, lane);
#pragma unroll
    for (int k = 0; k < PF; k++)
        if (t.z0 + 1 + k <= t.z1) load_row<DT, true>(q[k], Xc + (int64_t)(t.z0 + 1 + k - zx) * zs, 0, act, needL, needR, lane);
    load_row<DT, true>(ym, Xm + (int64_t)(t.z0 - zx) * zs, 0, act, false, false, lane);
    load_row<DT, true>(yp, Xp + (int64_t)(t.z0 - zx) * zs, 0, act, false, false, lane);

    const bool full = (x >= t.x0) && (x + VEC <= t.x1);
    for (int z = t.z0; z < t.z1; z++) {
        if (z + 1 < t.z1) {
            load_row<DT, true>(nym, Xm + (int64_t)(z + 1 - zx) * zs, 0, act, false, false, lane);
            load_row<DT, true>(nyp, Xp + (int64_t)(z + 1 - zx) * zs, 0, act, false, false, lane);
        }
        A left = __shfl_up_sync(0xffffffffu, zc.v[VEC - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, zc.v[0], 1);
        if (lane == 0) left = needL ? zc.l : A(1);
        if (lane == 31) right = needR ? zc.r : A(1);
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
            out[k] = s;
        }
        div6_n(out);
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
        if (nz <= t.z1) load_row<DT, true>(q[PF - 1], Xc + (int64_t)(nz - zx) * zs, 0, act, needL, needR, lane);
        ym = nym;
        yp = nyp;
    }
}

// ------------------------------------------------------------------------------------------
// CTA variant: one CTA of T threads (256 or 512) per tile of ny rows x nch 16-byte chunks of the
// work box, one chunk per thread (ny * nch <= T), marching z.  A box narrower than 32 chunks gets more rows per
// tile rather than idle lanes, and a wide box is cut into bands of equal width, so the lanes stay
// busy whatever the partition's shape.  Plane z' of the staged region -- rows y0-1 .. y0+ny and
// chunks xb-VEC .. xb+nch*VEC (the tile's chunks plus one halo chunk on each side, each halo chunk
// only where the tile's output range ends on a chunk boundary) -- is entry e = z' - z0 + 1 of the
// tile's plane sequence and goes into stage e % NS of a shared-memory ring by cp.async from every
// thread, so each input row is fetched once per CTA.  A step computes two output planes z, z+1
// from entries k .. k+3 (planes z-1 .. z+2, k = z - z0), after refilling the stages of entries k-2
// and k-1 (read by nobody since the barrier of this step) with entries k+NS-2 and k+NS-1: NS - 4
// planes stay in flight ahead of those being computed, and the barrier, the ring bookkeeping and
// the centre plane z+1 (also plane z's upper neighbour) are shared by the two outputs.  A stage is
// stage_slots >= (ny + 2) x (nch + 2) slots of 16 bytes, stage_slots <= 2T.  Tiles are ordered
// (z chunk, band, rows), so the CTAs resident together hold y-neighbouring tiles whose shared halo
// rows meet in L2.
// ------------------------------------------------------------------------------------------
template <int DT, int NS, int T>
__global__ void __launch_bounds__(T, 1024 / T) k_stencil3d_cta(const StenPart3D *__restrict__ parts,
                                                       const StenTile3D *__restrict__ tiles, int stage_slots,
                                                       const Seg *__restrict__ segs)
{
    static_assert((NS & (NS - 1)) == 0 && NS >= 6, "ring depth: a power of two, at least 6");
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    using V = typename EL::V;
    constexpr int VEC = EL::VEC;
    extern __shared__ uint4 smem[];
    const int lane = threadIdx.x & 31;
    const StenTile3D t = tiles[blockIdx.x];
    const StenPart3D P = parts[t.part];
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(smem);

    receive_segments_cta<E>(segs, t.seg0, t.nseg);

    const int ny = t.ny, nch = t.nch, rw = nch + 2;  // a staged row: halo chunk, nch chunks, halo chunk
    const int SS = (ny + 2) * rw;                     // 16-byte slots used per stage
    const int L = t.z1 - t.z0;                        // output planes; entries 0 .. L+1
    const int64_t zs = P.xs0, ys = P.xs1;
    const bool needL = t.x0 == t.xb;              // x0 - 1 lies in the left halo chunk
    const bool needR = t.x1 == t.xb + nch * VEC;  // x1 lies in the right halo chunk

    // This thread's copy items, fixed for the whole march: slots j and j + T of every plane.
    const int j0 = threadIdx.x, j1 = threadIdx.x + T;
    const int r0 = j0 / rw, c0 = j0 - r0 * rw, r1 = j1 / rw, c1 = j1 - r1 * rw;
    const bool has0 = j0 < SS && (c0 > 0 || needL) && (c0 < rw - 1 || needR);
    const bool has1 = j1 < SS && (c1 > 0 || needL) && (c1 < rw - 1 || needR);
    // entry e's slot (rr, cc) holds row y0 - 1 + rr, elements xb + (cc - 1) * VEC .. of plane z0 - 1 + e
    const E *src = reinterpret_cast<const E *>(P.x) + (int64_t)(t.z0 - 1 - P.xlo0) * zs +
                   (int64_t)(t.y - 1 - P.xlo1) * ys + (t.xb - VEC - P.xlo2);
    const int64_t g0 = (int64_t)r0 * ys + c0 * VEC, g1 = (int64_t)r1 * ys + c1 * VEC;
    const uint32_t stage_bytes = (uint32_t)stage_slots * 16u;
    int enext = 0;  // next entry to issue
    auto issue = [&]() {
        if (enext <= L + 1) {
            const uint32_t sb = ring_s + (uint32_t)(enext & (NS - 1)) * stage_bytes;
            if (has0) cpa16(sb + (uint32_t)j0 * 16u, src + g0);
            if (has1) cpa16(sb + (uint32_t)j1 * 16u, src + g1);
            src += zs;
        }
        enext++;
        cpa_commit();  // one group per entry, empty past the end
    };
#pragma unroll 1
    for (int k = 0; k < NS - 2; k++) issue();  // entries 0 .. NS-3

    // the chunk this thread computes: row r, chunk c (every chunk of the tile holds outputs)
    const int r = threadIdx.x / nch, c = threadIdx.x - r * nch;
    const int x = t.xb + c * VEC;
    const bool act = r < ny;
    const bool full = x >= t.x0 && x + VEC <= t.x1;
    const int me = (r + 1) * rw + c + 1;
    // x neighbours of the chunk's end elements: from the next lane's registers when it holds the
    // neighbouring chunk of the same row, else from the staged row (the halo chunks included)
    const bool shflL = c > 0 && lane > 0, shflR = c < nch - 1 && lane < 31;
    const bool haveL = c > 0 || needL, haveR = c < nch - 1 || needR;
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.y + r - P.ylo1) * P.ys1 + (x - P.ylo2) +
            (int64_t)(t.z0 - P.ylo0) * P.ys0;

    auto ld = [&](int e, int off, A (&v)[VEC]) {  // chunk `me + off` of entry e
        if (act) {
            EL::unpack(*reinterpret_cast<const V *>(smem + (e & (NS - 1)) * stage_slots + me + off), v);
        } else {
#pragma unroll
            for (int k = 0; k < VEC; k++) v[k] = A(1);  // idle threads: sums of ones
        }
    };
    // plane with centre cv (entry e), y neighbours from entry e, z neighbours zm and zq; stored at yq
    auto plane = [&](int e, const A (&cv)[VEC], const A (&zm)[VEC], const A (&zq)[VEC], E *out_p) {
        A ym[VEC], yq[VEC];
        ld(e, -rw, ym);
        ld(e, rw, yq);
        A left = __shfl_up_sync(0xffffffffu, cv[VEC - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, cv[0], 1);
        const E *row = reinterpret_cast<const E *>(smem + (e & (NS - 1)) * stage_slots + me);
        if (!shflL) left = act && haveL ? EL::load1(row - 1) : A(1);
        if (!shflR) right = act && haveR ? EL::load1(row + VEC) : A(1);
        A out[VEC];
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const A wv = k > 0 ? cv[k - 1] : left;
            const A ev = k < VEC - 1 ? cv[k + 1] : right;
            A s = wv + ev;
            s = s + ym[k];
            s = s + yq[k];
            s = s + zm[k];
            s = s + zq[k];
            out[k] = s;
        }
        div6_n(out);
        if (act) {
            if (full) {
                *reinterpret_cast<V *>(out_p) = EL::pack(out);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (x + k >= t.x0 && x + k < t.x1) EL::store1(out_p + k, out[k]);
            }
        }
    };

    for (int k = 0; k < L; k += 2) {
        cpa_wait<NS - 6>();  // entries up to k + 3 have landed (this thread's copies)
        __syncthreads();     // ... and every other thread's; the stages of k-2 and k-1 are free
        issue();             // entry k + NS - 2
        issue();             // entry k + NS - 1
        A zm[VEC], cv[VEC], zq[VEC];
        ld(k, 0, zm);
        ld(k + 1, 0, cv);
        ld(k + 2, 0, zq);
        plane(k + 1, cv, zm, zq, yp);  // output plane z0 + k
        if (k + 1 < L) {               // output plane z0 + k + 1: centre zq, below cv, above entry k+3
            A zq2[VEC];
            ld(k + 3, 0, zq2);
            plane(k + 2, zq, cv, zq2, yp + P.ys0);
        }
        yp += 2 * P.ys0;
    }
    cpa_wait<0>();
}

// ------------------------------------------------------------------------------------------
// The CTA variant with its planes staged by the tensor memory accelerator: the same tiles, ring
// and two output planes per step as above, but entry e (plane z0 - 1 + e of rows y0 - 1 ..
// y0 + ny and chunks xb - VEC .. of the part's X buffer) arrives as one bulk tensor copy
// (cp.async.bulk.tensor.3d) issued by thread 0 into its stage, completing a transaction-count
// mbarrier the computing threads wait on, instead of a cp.async per thread and slot.  The box
// of a part's tensor map is its tiles' staged plane (rwb chunks x boxh rows; a ragged tile loads
// rows it does not read, coordinates outside the buffer read zeros).  The receive phase's stores
// are ordinary (generic) writes to the X buffer, so every thread fences them to the async proxy
// before the barrier after which the first bulk copy is issued.  Waits are bounded: after
// spin_limit polls a wait gives up, the tile computes nothing, thread 0 waits (with a fixed limit)
// for the copies it issued and the error word is set.
// ------------------------------------------------------------------------------------------

template <int DT, int NS, int T>
__global__ void __launch_bounds__(T, 1024 / T) k_stencil3d_tma(const StenPart3D *__restrict__ parts,
                                                       const StenTile3D *__restrict__ tiles, int stage_slots,
                                                       const Seg *__restrict__ segs,
                                                       const uint8_t *__restrict__ tmaps, unsigned *err,
                                                       unsigned spin_limit)
{
    static_assert((NS & (NS - 1)) == 0 && NS >= 6, "ring depth: a power of two, at least 6");
    using EL = Elem<DT>;
    using E = typename EL::E;
    using A = typename EL::A;
    using V = typename EL::V;
    constexpr int VEC = EL::VEC;
    extern __shared__ uint4 smem_dyn[];
    __shared__ __align__(8) uint64_t full[NS];
    const int lane = threadIdx.x & 31;
    const StenTile3D t = tiles[blockIdx.x];
    const StenPart3D P = parts[t.part];
    // the ring starts on a 128-byte boundary (the launch adds 128 bytes of slack)
    const uint32_t ring_s = (smem_addr(smem_dyn) + 127u) & ~127u;
    const uint4 *ring = reinterpret_cast<const uint4 *>(reinterpret_cast<const char *>(smem_dyn) +
                                                          (ring_s - smem_addr(smem_dyn)));

    if (t.nseg > 0) receive_flat_vec<E>(segs, t.seg0, t.nseg, threadIdx.x, blockDim.x);
    asm volatile("fence.proxy.async.global;" ::: "memory");  // the receive's stores, before bulk copies read them
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int ny = t.ny, nch = t.nch, rw = P.rwb;  // a staged row: halo chunk, nch chunks, halo chunk(s)
    const int L = t.z1 - t.z0;                      // output planes; entries 0 .. L+1
    const bool needL = t.x0 == t.xb;              // x0 - 1 lies in the left halo chunk
    const bool needR = t.x1 == t.xb + nch * VEC;  // x1 lies in the right halo chunk
    const uint32_t stage_bytes = (uint32_t)stage_slots * 16u;
    const uint32_t box_bytes = (uint32_t)P.boxh * (uint32_t)rw * 16u;
    const uint8_t *tmap = tmaps + (size_t)t.part * 128;
    const int xc = (int)(t.xb - VEC - P.xlo2), yc = (int)(t.y - 1 - P.xlo1), zc = (int)(t.z0 - 1 - P.xlo0);
    int issued = 0;  // thread 0: entries issued so far
    auto issue = [&](int e) {
        if (e > L + 1) return;
        const uint32_t bar = smem_addr(&full[e & (NS - 1)]);
        const uint32_t dst = ring_s + (uint32_t)(e & (NS - 1)) * stage_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(box_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
            "l"(tmap), "r"(xc), "r"(yc), "r"(zc + e), "r"(bar)
            : "memory");
        issued = e + 1;
    };
    if (threadIdx.x == 0)
        for (int e = 0; e < NS - 2; e++) issue(e);  // entries 0 .. NS-3

    // the chunk this thread computes: row r, chunk c (every chunk of the tile holds outputs)
    const int r = threadIdx.x / nch, c = threadIdx.x - r * nch;
    const int x = t.xb + c * VEC;
    const bool act = r < ny;
    const bool full_chunk = x >= t.x0 && x + VEC <= t.x1;
    const int me = (r + 1) * rw + c + 1;
    const bool shflL = c > 0 && lane > 0, shflR = c < nch - 1 && lane < 31;
    const bool haveL = c > 0 || needL, haveR = c < nch - 1 || needR;
    E *yp = reinterpret_cast<E *>(P.y) + (int64_t)(t.y + r - P.ylo1) * P.ys1 + (x - P.ylo2) +
            (int64_t)(t.z0 - P.ylo0) * P.ys0;

    auto ld = [&](int e, int off, A (&v)[VEC]) {  // chunk `me + off` of entry e
        if (act) {
            EL::unpack(*reinterpret_cast<const V *>(ring + (e & (NS - 1)) * stage_slots + me + off), v);
        } else {
#pragma unroll
            for (int k = 0; k < VEC; k++) v[k] = A(1);  // idle threads: sums of ones
        }
    };
    auto plane = [&](int e, const A (&cv)[VEC], const A (&zm)[VEC], const A (&zq)[VEC], E *out_p) {
        A ym[VEC], yq[VEC];
        ld(e, -rw, ym);
        ld(e, rw, yq);
        A left = __shfl_up_sync(0xffffffffu, cv[VEC - 1], 1);
        A right = __shfl_down_sync(0xffffffffu, cv[0], 1);
        const E *row = reinterpret_cast<const E *>(ring + (e & (NS - 1)) * stage_slots + me);
        if (!shflL) left = act && haveL ? EL::load1(row - 1) : A(1);
        if (!shflR) right = act && haveR ? EL::load1(row + VEC) : A(1);
        A out[VEC];
#pragma unroll
        for (int k = 0; k < VEC; k++) {
            const A wv = k > 0 ? cv[k - 1] : left;
            const A ev = k < VEC - 1 ? cv[k + 1] : right;
            A s = wv + ev;
            s = s + ym[k];
            s = s + yq[k];
            s = s + zm[k];
            s = s + zq[k];
            out[k] = s;
        }
        div6_n(out);
        if (act) {
            if (full_chunk) {
                *reinterpret_cast<V *>(out_p) = EL::pack(out);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; k++)
                    if (x + k >= t.x0 && x + k < t.x1) EL::store1(out_p + k, out[k]);
            }
        }
    };

    bool failed = false;
    for (int k = 0; k < L; k += 2) {
        // entries k .. k+3 must have landed; the earlier ones were waited for in earlier steps
        bool ok = true;
        for (int e = k == 0 ? 0 : k + 2; e <= k + 3 && e <= L + 1; e++)
            ok = ok && mbar_wait_bounded(smem_addr(&full[e & (NS - 1)]), (uint32_t)((e / NS) & 1), spin_limit);
        // every thread is done with the stages of entries k-2 and k-1; a failed wait anywhere
        // stops every thread
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (threadIdx.x == 0) {
            issue(k + NS - 2);
            issue(k + NS - 1);
        }
        A zm[VEC], cv[VEC], zq[VEC];
        ld(k, 0, zm);
        ld(k + 1, 0, cv);
        ld(k + 2, 0, zq);
        plane(k + 1, cv, zm, zq, yp);  // output plane z0 + k
        if (k + 1 < L) {               // output plane z0 + k + 1: centre zq, below cv, above entry k+3
            A zq2[VEC];
            ld(k + 3, 0, zq2);
            plane(k + 2, zq, cv, zq2, yp + P.ys0);
        }
        yp += 2 * P.ys0;
    }
    if (failed && threadIdx.x == 0) {
        // the copies issued land before the CTA's shared memory is released: the last one of each
        // stage completes that stage's latest phase
        for (int e = issued - 1; e >= 0 && e >= issued - NS; e--)
            mbar_wait_bounded(smem_addr(&full[e & (NS - 1)]), (uint32_t)((e / NS) & 1), TMA_DRAIN_LIMIT);
        if (err) atomicOr(err, 1u);
    }
}

cudaError_t launch_stencil3d(int dtype, const StenPart3D *parts, const StenTile3D *tiles,
                             int ntiles, const Seg *segs, int warps_per_cta, int variant, size_t smem,
                             cudaStream_t s, const void *tmaps, unsigned *err, unsigned spin_limit)
{
    if (ntiles <= 0) return cudaSuccess;
    if (variant == 3) {
        constexpr int NS = STENCIL3D_STAGES;
        const int T = warps_per_cta == 16 ? 512 : 256;
        if (!tmaps || smem < 128) return cudaErrorInvalidValue;
        const int slots = (int)((smem - 128) / ((size_t)NS * 16));
        if (slots < 1 || slots % 8 != 0 || smem != (size_t)NS * slots * 16 + 128) return cudaErrorInvalidValue;
        const int which = (dtype == DT_F64 ? 0 : dtype == DT_F32 ? 1 : dtype == DT_BF16 ? 2 : -1);
        if (which < 0) return cudaErrorInvalidValue;
        using KFn = void (*)(const StenPart3D *, const StenTile3D *, int, const Seg *, const uint8_t *, unsigned *,
                             unsigned);
        const KFn fns[2][3] = {{k_stencil3d_tma<DT_F64, NS, 256>, k_stencil3d_tma<DT_F32, NS, 256>, k_stencil3d_tma<DT_BF16, NS, 256>},
                               {k_stencil3d_tma<DT_F64, NS, 512>, k_stencil3d_tma<DT_F32, NS, 512>, k_stencil3d_tma<DT_BF16, NS, 512>}};
        const int wt = T == 512 ? 1 : 0;
        static bool attr[2][3] = {};
        if (!attr[wt][which]) {
            cudaError_t e = cudaFuncSetAttribute(fns[wt][which], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 NS * 768 * 16 + 128);
            if (e != cudaSuccess) return e;
            attr[wt][which] = true;
        }
        if (smem > (size_t)NS * 768 * 16 + 128) return cudaErrorInvalidValue;
        fns[wt][which]<<<ntiles, T, smem, s>>>(parts, tiles, slots, segs, reinterpret_cast<const uint8_t *>(tmaps), err,
                                               spin_limit);
        return cudaGetLastError();
    }
    if (variant == 1) {
        constexpr int NS = STENCIL3D_STAGES;
        const int T = warps_per_cta == 16 ? 512 : 256;
        const int slots = (int)(smem / ((size_t)NS * 16));
        if (slots < 1 || slots > 2 * T || smem != (size_t)NS * slots * 16) return cudaErrorInvalidValue;
        const int which = (dtype == DT_F64 ? 0 : dtype == DT_F32 ? 1 : dtype == DT_BF16 ? 2 : -1);
        if (which < 0) return cudaErrorInvalidValue;
        using KFn = void (*)(const StenPart3D *, const StenTile3D *, int, const Seg *);
        const KFn fns[2][3] = {{k_stencil3d_cta<DT_F64, NS, 256>, k_stencil3d_cta<DT_F32, NS, 256>, k_stencil3d_cta<DT_BF16, NS, 256>},
                               {k_stencil3d_cta<DT_F64, NS, 512>, k_stencil3d_cta<DT_F32, NS, 512>, k_stencil3d_cta<DT_BF16, NS, 512>}};
        const int wt = T == 512 ? 1 : 0;
        static bool attr[2][3] = {};
        if (!attr[wt][which]) {
            cudaError_t e = cudaFuncSetAttribute(fns[wt][which], cudaFuncAttributeMaxDynamicSharedMemorySize, NS * 2 * T * 16);
            if (e != cudaSuccess) return e;
            attr[wt][which] = true;
        }
        fns[wt][which]<<<ntiles, T, smem, s>>>(parts, tiles, slots, segs);
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
