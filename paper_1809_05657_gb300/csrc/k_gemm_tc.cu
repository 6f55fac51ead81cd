// k_gemm_tc.cu -- the GEMM of Listing 3 (C = beta*C + alpha*A*B, A optionally lower triangular)
// on binary32 arrays, computed on the 5th-generation tensor cores in bfloat16 with the "bf16x3"
// split of Henry, Tang & Heinecke (ARITH 2019): every operand is split into x = hi + lo with
// hi = bf16(x) and lo = bf16(x - hi), and A*B is accumulated in binary32 as
// Ahi*Bhi + Ahi*Blo + Alo*Bhi (the lo*lo term is dropped).  Each bf16 x bf16 product is exact in
// binary32; what remains is the representation error of the split (about 2^-17 relative per
// operand), the dropped term (about 2^-18) and the binary32 accumulation.
//
// One CTA (256 threads) computes a 128 x 256 tile of C:
//   * all threads load the binary32 A (128 x 64) and B (64 x 256) slices of the next K step,
//     split them and store hi and lo parts into shared memory in the canonical K-major layout with
//     the 128-byte swizzle (row r at r*128 bytes, 16-byte chunk c stored at chunk c ^ (r % 8));
//   * one thread issues the tcgen05.mma instructions (M=128, N=256, K=16 each, three per K=16
//     slice) into a binary32 accumulator in tensor memory (256 columns) and commits them to an
//     mbarrier; the next slice is split into the other of two stages meanwhile;
//   * at the end every warp reads its 32 rows x 128 columns of the accumulator back with
//     tcgen05.ld and writes C.
// Triangular A: a tile of rows [i0, i0+128) needs K only up to i0+128, and elements above the
// diagonal are never read.  Tiles are launched heaviest first.
//
// Every wait on an mbarrier is bounded; a wait that gives up sets *err, stops issuing work,
// waits (bounded) for the tensor core work already committed, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hda {

namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int A_BYTES = BM * BK * 2;       // one bf16 part of the A slice: 16 KB
constexpr int B_BYTES = BN * BK * 2;       // one bf16 part of the B slice: 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // hi + lo of A and B: 96 KB
constexpr int TMEM_COLS = 256;
constexpr unsigned WAIT_LIMIT = 1u << 24;  // polls (with a short sleep) before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D binary32, A and B bfloat16, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit = WAIT_LIMIT)
{
    for (unsigned i = 0; i < limit; i++) {
        if (mbar_try(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

// bf16 hi / lo split of one binary32 value
__device__ __forceinline__ void split(float x, uint16_t &h, uint16_t &l)
{
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r = x - __bfloat162float(bh);
    h = __bfloat16_as_ushort(bh);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(r));
}

// Byte offset of 16-byte chunk c of row r in a K-major 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// The same for the 64-byte swizzle (rows of 64 bytes, 32 bf16 of K): chunk c of row r stored at
// chunk c ^ ((r / 2) % 4), the pattern repeating every 8 rows (512 bytes).
__device__ __forceinline__ uint32_t sw64_off(int r, int c) { return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4)); }

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

}  // namespace

__global__ void __launch_bounds__(256, 1) k_gemm_bf16x3(const TcPart *__restrict__ parts,
                                                        const TcTile *__restrict__ tiles, float alpha,
                                                        float beta, unsigned *err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t taddr_s;
    __shared__ int abort_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TcTile tile = tiles[blockIdx.x];
    const TcPart P = parts[tile.part];
    const float *A = reinterpret_cast<const float *>(P.a);
    const float *B = reinterpret_cast<const float *>(P.b);
    float *C = reinterpret_cast<float *>(P.c);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        abort_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = taddr_s;

    const int i0 = tile.i0, j0 = tile.j0;
    const int nkt = (tile.kend + BK - 1) / BK;
    uint32_t phase[2] = {0u, 0u};
    int issued[2] = {0, 0};  // a commit to this stage's barrier is outstanding
    for (int kt = 0; kt < nkt; kt++) {
        const int s = kt & 1;
        if (issued[s]) {  // the MMAs that read this stage (two slices ago) must be done
            if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) abort_s = 1;
            phase[s] ^= 1u;
            issued[s] = 0;
        }
        __syncthreads();
        if (abort_s) break;
        uint8_t *st = smem + s * STAGE_BYTES;
        uint8_t *ahi = st, *alo = st + A_BYTES, *bhi = st + 2 * A_BYTES, *blo = st + 2 * A_BYTES + B_BYTES;
        const int k0 = kt * BK;
        // A slice: a warp per row (lanes along K, coalesced loads), 2-byte swizzled stores
        for (int r = warp; r < BM; r += 8) {
            const int i = i0 + r;
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int kl = half * 32 + lane, k = k0 + kl;
                float v = 0.0f;
                if (i < P.i1 && k < tile.kend && (!P.lower || k <= i))
                    v = A[(int64_t)(i - P.alo0) * P.as + (k - P.alo1)];
                uint16_t h, l;
                split(v, h, l);
                const uint32_t off = sw_off(r, kl >> 3) + ((kl & 7) << 1);
                *reinterpret_cast<uint16_t *>(ahi + off) = h;
                *reinterpret_cast<uint16_t *>(alo + off) = l;
            }
        }
        // B slice: stored transposed (row n, 64 k); thread -> column n, chunks of 8 k
        {
            const int n = tid;  // BN == 256 == blockDim.x
            const int j = j0 + n;
            for (int c = 0; c < 8; c++) {
                uint16_t h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const int k = k0 + c * 8 + e;
                    float v = 0.0f;
                    if (j < P.j1 && k < tile.kend) v = B[(int64_t)(k - P.blo0) * P.bs + (j - P.blo1)];
                    split(v, h[e], l[e]);
                }
                uint4 H, L;
                H.x = h[0] | ((uint32_t)h[1] << 16); H.y = h[2] | ((uint32_t)h[3] << 16);
                H.z = h[4] | ((uint32_t)h[5] << 16); H.w = h[6] | ((uint32_t)h[7] << 16);
                L.x = l[0] | ((uint32_t)l[1] << 16); L.y = l[2] | ((uint32_t)l[3] << 16);
                L.z = l[4] | ((uint32_t)l[5] << 16); L.w = l[6] | ((uint32_t)l[7] << 16);
                *reinterpret_cast<uint4 *>(bhi + sw_off(n, c)) = H;
                *reinterpret_cast<uint4 *>(blo + sw_off(n, c)) = L;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(ahi), a_lo = smem_u32(alo), b_hi = smem_u32(bhi), b_lo = smem_u32(blo);
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++) {
                const uint32_t off = kk * 32;  // 16 bf16 along K inside the 128-byte swizzle row
                mma_bf16(tmem, sw128_desc(a_hi + off), sw128_desc(b_hi + off), (kt > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(tmem, sw128_desc(a_hi + off), sw128_desc(b_lo + off), 1u);
                mma_bf16(tmem, sw128_desc(a_lo + off), sw128_desc(b_hi + off), 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[s]))
                         : "memory");
        }
        issued[s] = 1;
    }
    // wait for every committed slice (bounded even after an abort, so no MMA is left running)
    bool ok = !abort_s;
    for (int s = 0; s < 2; s++) {
        if (issued[s]) {
            if (!mbar_wait(smem_u32(&mbar[s]), phase[s])) ok = false;
            phase[s] ^= 1u;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (abort_s) ok = false;
    if (ok && nkt > 0) {
        // epilogue: warp w reads lanes 32*(w%4).. (rows) and columns (w/4)*128 .. +127
        const int lane_base = 32 * (warp & 3);
        const int col_base = 128 * (warp >> 2);
        const int i = i0 + lane_base + lane;
        for (int cc = 0; cc < 4; cc++) {
            uint32_t r[32];
            const uint32_t ta = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(col_base + cc * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                  "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                  "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                  "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (i < P.i1) {
                float *crow = C + (int64_t)(i - P.clo0) * P.cs;
#pragma unroll
                for (int e = 0; e < 32; e++) {
                    const int j = j0 + col_base + cc * 32 + e;
                    if (j < P.j1) {
                        float *cp = crow + (j - P.clo1);
                        const float acc = __uint_as_float(r[e]);
                        *cp = beta == 0.0f ? alpha * acc : beta * *cp + alpha * acc;
                    }
                }
            }
        }
    } else if (tid == 0 && !ok) {
        atomicOr(err, 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

size_t gemm_tc_smem_bytes() { return 2 * (size_t)STAGE_BYTES + 1024; }

cudaError_t launch_gemm_tc(const TcPart *parts, const TcTile *tiles, int ntiles, float alpha, float beta,
                           unsigned *err, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    static bool attr = false;
    const size_t sm = gemm_tc_smem_bytes();
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_gemm_bf16x3<<<ntiles, 256, sm, s>>>(parts, tiles, alpha, beta, err);
    return cudaGetLastError();
}



// ==========================================================================================
// Pre-split operand panels and the pipelined tensor-core GEMM.
//
// Panels: the bf16 parts of A (per device, its 128-row tiles) and of B^T (column tiles of the
// CTA width, 256), each 128 x BKp (A) or 256 x BKp (B) tile stored contiguously in exactly the
// K-major swizzled layout the MMA reads, so a K step of a CTA is two contiguous bulk copies.
// With NSP parts per operand (2: hi, lo -- "bf16x3", BKp = 64, 128-byte rows and swizzle; 3: hi,
// mid, lo -- "bf16x6", BKp = 32, 64-byte rows and swizzle), a panel tile (mt, kt) part q sits at
// ((mt * nkt + kt) * NSP + q) * 128 * BKp * 2 and a B panel tile (nt, kt) part q at
// ((nt * nkt + kt) * NSP + q) * 256 * BKp * 2.
//
// bf16x6 (the same paper's higher-accuracy form): x = hi + mid + lo with hi = bf16(x),
// mid = bf16(x - hi), lo = bf16(x - hi - mid) (both differences exact in binary32), and the six
// products whose magnitude is at least about 2^-16 of a*b are kept: hi*hi, hi*mid, mid*hi, hi*lo,
// mid*mid, lo*hi.  The split leaves about 2^-24 of each operand and the dropped products
// (mid*lo, lo*mid, lo*lo) about 2^-23 of a*b, so the result is as accurate as binary32 products.
// Its CTA tile is 128 x 128 (three parts of A and of B fill the same 96 KB stage as two parts of
// a 128 x 256 tile).
// ==========================================================================================

namespace {

// bf16 hi / mid / lo split of one binary32 value
__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l)
{
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bm);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

__device__ __forceinline__ uint4 pack8(const uint16_t *v)
{
    uint4 u;
    u.x = v[0] | ((uint32_t)v[1] << 16); u.y = v[2] | ((uint32_t)v[3] << 16);
    u.z = v[4] | ((uint32_t)v[5] << 16); u.w = v[6] | ((uint32_t)v[7] << 16);
    return u;
}

// One CTA per (tile, part set): thread -> 16-byte chunk (row r, 8 consecutive k), every part.
// Tiles of bk = 64 k are 128-byte rows in the 128-byte swizzle, tiles of bk = 32 64-byte rows in the
// 64-byte swizzle.
__global__ void __launch_bounds__(256) k_split_panel(const SplitJob *__restrict__ jobs)
{
    const SplitJob J = jobs[blockIdx.y];
    const int tiles_per_row = J.nkt;  // k tiles per row tile
    const int tile = blockIdx.x;      // row tile * nkt + k tile
    if (tile >= J.ntiles) return;
    const int mt = tile / tiles_per_row, kt = tile - mt * tiles_per_row;
    const int rows = J.rows_per_tile;  // 128 (A) or the CTA width (B): powers of two
    const int nsp = J.nparts;          // 2 or 3
    const int bk = J.bk;               // 64 or 32
    const int cpr = bk / 8;            // 16-byte chunks per row
    const float *src = reinterpret_cast<const float *>(J.src);
    uint8_t *part0 = reinterpret_cast<uint8_t *>(J.dst) + (size_t)tile * nsp * rows * (bk * 2);
    for (int q = threadIdx.x; q < rows * cpr; q += blockDim.x) {
        const int r = J.transpose ? (q & (rows - 1)) : (q / cpr);
        const int c = J.transpose ? (q / rows) : (q - (q / cpr) * cpr);
        const int row = J.row0 + mt * rows + r;  // A: row i; B: column n
        uint16_t h[8], m[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int k = kt * bk + c * 8 + e;
            float v = 0.0f;
            if (row < J.row_end && k < J.kend && (!J.lower || k <= row)) {
                if (J.transpose) v = src[(int64_t)(k - J.lo0) * J.stride + (row - J.lo1)];  // B[k][n]
                else v = src[(int64_t)(row - J.lo0) * J.stride + (k - J.lo1)];             // A[i][k]
            }
            if (nsp == 3) split3(v, h[e], m[e], l[e]);
            else split(v, h[e], l[e]);
        }
        const uint32_t off = bk == 64 ? sw_off(r, c) : sw64_off(r, c);
        const size_t pb = (size_t)rows * bk * 2;
        *reinterpret_cast<uint4 *>(part0 + off) = pack8(h);
        if (nsp == 3) {
            *reinterpret_cast<uint4 *>(part0 + pb + off) = pack8(m);
            *reinterpret_cast<uint4 *>(part0 + 2 * pb + off) = pack8(l);
        } else {
            *reinterpret_cast<uint4 *>(part0 + pb + off) = pack8(l);
        }
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

constexpr int P_STAGES_MAX = 3;

// Panel GEMM geometry for NSP bf16 parts per operand.  Both forms compute 128 x 256 tiles of C.
// bf16x3: K steps of 64 (128-byte rows, 128-byte swizzle), two stages of 96 KB.  bf16x6: K steps
// of 32 (64-byte rows, 64-byte swizzle), three stages of 72 KB -- the same MMA work per stage as a
// 128 x 128 tile with K steps of 64, and a quarter fewer operand bytes streamed per MMA flop.
template <int NSP>
struct PanelGeo {
    static constexpr int BNp = 256;                                 // CTA tile width
    static constexpr int BKp = NSP == 3 ? 32 : 64;                  // K per stage
    static constexpr int STAGES = NSP == 3 ? 3 : 2;
    static constexpr int A_BYTESp = BM * BKp * 2;                   // one part of the A slice
    static constexpr int B_BYTESp = BNp * BKp * 2;                  // one part of the B slice
    static constexpr int STAGEp = NSP * A_BYTESp + NSP * B_BYTESp;  // 96 KB (x3), 72 KB (x6)
    static constexpr uint32_t IDESCp = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BNp >> 3) << 17) |
                                       ((uint32_t)(BM >> 4) << 24);
    __device__ static uint64_t desc(uint32_t saddr) { return NSP == 3 ? sw64_desc(saddr) : sw128_desc(saddr); }
};
static_assert(PanelGeo<2>::STAGEp == STAGE_BYTES && PanelGeo<3>::STAGEp == 72 * 1024, "stage size");
static_assert(PanelGeo<2>::STAGES * PanelGeo<2>::STAGEp + 1024 <= 227 * 1024 &&
              PanelGeo<3>::STAGES * PanelGeo<3>::STAGEp + 1024 <= 227 * 1024, "shared memory");
static_assert(PanelGeo<3>::STAGES <= P_STAGES_MAX && PanelGeo<2>::STAGES <= P_STAGES_MAX, "stages");

__device__ __forceinline__ void mma_bf16_id(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

}  // namespace

// Warp-specialised GEMM: warp 0 lane 0 streams panel tiles into a two-stage ring with bulk copies
// (full barriers carry the byte count), warp 1 lane 0 issues the MMAs and commits each stage back
// to its empty barrier and the final result to the done barrier, warps 4..7 read the accumulator
// from tensor memory and write C.  Every wait is bounded: the ring's waits give up after
// spin_limit polls (the library's setting), and then the producer waits -- with the fixed limit --
// for the bulk copies it has issued, the MMAs already issued complete before the tensor memory is
// released, the tile's C is left alone and the error word is set.
template <int NSP>
__global__ void __launch_bounds__(256, 1) k_gemm_bf16x3_panels(const PanelPart *__restrict__ parts,
                                                               const TcTile *__restrict__ tiles, float alpha,
                                                               float beta, unsigned *err, unsigned spin_limit)
{
    using G = PanelGeo<NSP>;
    constexpr int BNp = G::BNp;
    constexpr uint32_t TMEM_COLSp = (uint32_t)BNp;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int P_STAGES = G::STAGES;
    __shared__ __align__(8) uint64_t full[P_STAGES_MAX], empty[P_STAGES_MAX], done;
    __shared__ uint32_t taddr_s;
    __shared__ volatile int fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const TcTile tile = tiles[blockIdx.x];
    const PanelPart P = parts[tile.part];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(TMEM_COLSp)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < P_STAGES; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = taddr_s;
    const int nkt = (tile.kend + G::BKp - 1) / G::BKp;
    const int mt = (tile.i0 - P.row0) / BM, nt = (tile.j0 - P.col0) / BNp;

    if (warp == 0 && lane == 0) {  // producer
        uint32_t ph[P_STAGES] = {};
        int fills[P_STAGES] = {};
        for (int kt = 0; kt < nkt && !fail; kt++) {
            const int s = kt % P_STAGES;
            if (kt >= P_STAGES) {
                if (!mbar_wait(smem_u32(&empty[s]), ph[s], spin_limit)) { fail = 1; break; }
                ph[s] ^= 1u;
            }
            fills[s]++;
            uint8_t *st = smem + s * G::STAGEp;
            const uint8_t *ap = reinterpret_cast<const uint8_t *>(P.apanel) + (size_t)((mt * P.nkt + kt) * NSP) * G::A_BYTESp;
            const uint8_t *bp = reinterpret_cast<const uint8_t *>(P.bpanel) + (size_t)((nt * P.nkt_b + kt) * NSP) * G::B_BYTESp;
            const uint32_t fb = smem_u32(&full[s]);
            mbar_expect(fb, (uint32_t)G::STAGEp);
            bulk_g2s(smem_u32(st), ap, NSP * G::A_BYTESp, fb);                     // every part of A
            bulk_g2s(smem_u32(st + NSP * G::A_BYTESp), bp, NSP * G::B_BYTESp, fb);  // every part of B
        }
        if (fail)  // every bulk copy issued lands before the CTA's shared memory is released
            for (int s = 0; s < P_STAGES; s++)
                if (fills[s] > 0) mbar_wait(smem_u32(&full[s]), (uint32_t)((fills[s] - 1) & 1));
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        uint32_t ph[P_STAGES] = {};
        int kt = 0;
        for (; kt < nkt && !fail; kt++) {
            const int s = kt % P_STAGES;
            if (!mbar_wait(smem_u32(&full[s]), ph[s], spin_limit)) { fail = 1; break; }
            ph[s] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = smem_u32(smem + s * G::STAGEp);
            const uint32_t a0 = st, b0 = st + NSP * G::A_BYTESp;  // part q at + q * A_BYTESp / B_BYTESp
#pragma unroll
            for (int kk = 0; kk < G::BKp / 16; kk++) {
                const uint32_t off = kk * 32;  // 16 bf16 of K along the (swizzled) row
                // (A part, B part) pairs: x3 keeps (0,0) (0,1) (1,0); x6 adds (0,2) (1,1) (2,0)
#pragma unroll
                for (int pr = 0; pr < (NSP == 3 ? 6 : 3); pr++) {
                    const int qa = pr == 2 ? 1 : pr == 4 ? 1 : pr == 5 ? 2 : 0;
                    const int qb = pr == 1 ? 1 : pr == 3 ? 2 : pr == 4 ? 1 : 0;
                    mma_bf16_id(tmem, G::desc(a0 + qa * G::A_BYTESp + off), G::desc(b0 + qb * G::B_BYTESp + off),
                                G::IDESCp, (kt > 0 || kk > 0 || pr > 0) ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        // the done barrier completes when every MMA issued above has finished
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    // everyone: wait for the accumulator (bounded; after a failure the MMAs already issued still
    // complete before the tensor memory is released)
    const bool ok = mbar_wait(smem_u32(&done), 0u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp >= 4 && ok && !fail && nkt > 0) {
        const int lane_base = 32 * (warp & 3);
        const int i = tile.i0 + lane_base + lane;
        float *C = reinterpret_cast<float *>(P.c);
        for (int cc = 0; cc < BNp / 32; cc++) {
            uint32_t r[32];
            const uint32_t ta = tmem + ((uint32_t)lane_base << 16) + (uint32_t)(cc * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                  "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                  "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                  "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (i < P.i1) {
                float *crow = C + (int64_t)(i - P.clo0) * P.cs;
#pragma unroll
                for (int e = 0; e < 32; e++) {
                    const int j = tile.j0 + cc * 32 + e;
                    if (j < P.j1 && (!P.upper || j >= i)) {
                        float *cp = crow + (j - P.clo1);
                        const float acc = __uint_as_float(r[e]);
                        *cp = beta == 0.0f ? alpha * acc : beta * *cp + alpha * acc;
                    }
                }
            }
        }
    }
    if (tid == 0 && (!ok || fail)) atomicOr(err, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLSp) : "memory");
}

cudaError_t launch_split_panels(const SplitJob *jobs, int njobs, int max_tiles, cudaStream_t s)
{
    if (njobs <= 0 || max_tiles <= 0) return cudaSuccess;
    dim3 grid(max_tiles, njobs);
    k_split_panel<<<grid, 256, 0, s>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_gemm_panels(const PanelPart *parts, const TcTile *tiles, int ntiles, float alpha,
                               float beta, unsigned *err, unsigned spin_limit, int nparts, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (nparts != 2 && nparts != 3) return cudaErrorInvalidValue;
    static bool attr[2] = {false, false};
    const size_t sm = nparts == 3 ? (size_t)PanelGeo<3>::STAGES * PanelGeo<3>::STAGEp + 1024
                                  : (size_t)PanelGeo<2>::STAGES * PanelGeo<2>::STAGEp + 1024;
    auto fn = nparts == 3 ? k_gemm_bf16x3_panels<3> : k_gemm_bf16x3_panels<2>;
    if (!attr[nparts - 2]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr[nparts - 2] = true;
    }
    fn<<<ntiles, 256, sm, s>>>(parts, tiles, alpha, beta, err, spin_limit);
    return cudaGetLastError();
}

}  // namespace hda
