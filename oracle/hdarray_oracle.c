/*
 * hdarray_oracle.c -- plain, slow CPU oracle for the HDArray hot path.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file's library. The GPU library never links, loads or calls it, and the two
 * share no code.
 *
 * What is computed here, from Cho, Kwon & Midkiff, "HDArray: Parallel Array Interface for
 * Distributed Heterogeneous Devices":
 *
 *   - Sections as per-element membership predicates: boxes ([LB:UB], Sec. 2.1), offset clauses
 *     composed with a work region (Sec. 3, "Offset clauses"), trapezoids (Sec. 3.1,
 *     HDArraySetTrapezoidUse/Def) and the even ROW/COL/BLOCK work partitions (Sec. 3.1,
 *     HDArrayPartition).
 *   - The communication that Eq. 1-4 (Sec. 2.2) produce, computed element by element on ONE
 *     unpartitioned index space: every element carries its last writer ("owner") and, per device,
 *     a flag "this device holds the current value".  sGDEF_{p,q} is then exactly the set of
 *     elements owned by p that q does not hold, and rGDEF_{p,q} = sGDEF_{q,p}.  A use of element e
 *     by device p that does not hold e is one message owner(e) -> p (Eq. 1 and 2); a definition by p
 *     makes p the owner and every other device stale (Eq. 3 and 4, with the last writer winning:
 *     a later definition by another device also removes the element from the older writer's
 *     sGDEF -- the paper only states that the runtime knows where the last written copy is, Sec. 1,
 *     and that GDEF says who owns the coherent copy, Sec. 3.1).
 *   - The workloads, evaluated on one global array: the Jacobi step of Sec. 5, a 3-D 7-point
 *     analogue, the GEMM of Listing 3, an element-wise squared difference, and the reductions of
 *     HDArrayReduce (Table 2).
 *
 * Floating point: binary64 unless a function says otherwise.  "prec" selects the storage type of
 * a stencil field: 0 = binary64, 1 = binary32, 2 = bfloat16 storage with binary32 arithmetic.
 * Build with -ffp-contract=off so that no multiply-add is fused behind the source's back.
 *
 * Coordinates: up to three dimensions, row-major, dimension 0 outermost.  Unused dimensions have
 * extent 1.  All ranges are half-open [lo, hi), except trapezoid corners, which name elements.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ALL INT32_MIN /* the '*' offset: every element of that dimension (Sec. 3) */

/* Threads of the stencil value loops (orc_jacobi2d, orc_stencil3d).  Every output element is a
 * function of the input array alone, so the loops give the same bits with any number of threads;
 * the default is one.  Without OpenMP at build time the loops always run on one thread. */
static int orc_nthreads = 1;

/* Set the value loops' thread count (clamped to >= 1); returns the count the loops will use. */
int orc_set_threads(int n)
{
    orc_nthreads = n < 1 ? 1 : n;
#ifdef _OPENMP
    return orc_nthreads;
#else
    orc_nthreads = 1;
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------------ */
/* Partitions: HDArrayPartition splits a work region evenly over the devices (Sec. 3.1).        */
/* ------------------------------------------------------------------------------------------ */

/* Even split of [a, b) into P blocks; block p.  The first (b - a) mod P blocks get one extra
 * element, so block sizes differ by at most one. */
static void split_even(int64_t a, int64_t b, int P, int p, int64_t *lo, int64_t *hi)
{
    int64_t n = b - a;
    int64_t q = n / P;
    int64_t m = n % P;
    int64_t extra_before = p < m ? p : m;
    *lo = a + (int64_t)p * q + extra_before;
    *hi = *lo + q + (p < m ? 1 : 0);
}

/* BLOCK uses a Pr x Pc grid of devices with Pr the largest divisor of P with Pr*Pr <= P. */
static void block_grid(int P, int *Pr, int *Pc)
{
    int r = 1;
    for (int d = 1; d * d <= P; d++)
        if (P % d == 0) r = d;
    *Pr = r;
    *Pc = P / r;
}

/* Work box of device p for partition type (0 ROW: split dimension 0, "the highest dimension",
 * Sec. 3.2; 1 COL: split dimension 1; 2 BLOCK: split dimensions 0 and 1 on the device grid,
 * device p at grid row p / Pc, grid column p % Pc).  Returns 0, or -1 for an invalid request. */
int orc_partition_box(int type, int P, int p, int dim, const int64_t *rlo, const int64_t *rhi,
                      int64_t *lo, int64_t *hi)
{
    if (P < 1 || p < 0 || p >= P || dim < 1 || dim > 3) return -1;
    for (int d = 0; d < 3; d++) {
        lo[d] = d < dim ? rlo[d] : 0;
        hi[d] = d < dim ? rhi[d] : 1;
    }
    if (type == 0) {
        split_even(rlo[0], rhi[0], P, p, &lo[0], &hi[0]);
    } else if (type == 1) {
        if (dim < 2) return -1;
        split_even(rlo[1], rhi[1], P, p, &lo[1], &hi[1]);
    } else if (type == 2) {
        if (dim < 2) return -1;
        int Pr, Pc;
        block_grid(P, &Pr, &Pc);
        split_even(rlo[0], rhi[0], Pr, p / Pc, &lo[0], &hi[0]);
        split_even(rlo[1], rhi[1], Pc, p % Pc, &lo[1], &hi[1]);
    } else {
        return -1;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Membership predicates, one element at a time.                                                */
/* ------------------------------------------------------------------------------------------ */

static int in_bounds(const int64_t *n, const int64_t *e)
{
    for (int d = 0; d < 3; d++)
        if (e[d] < 0 || e[d] >= n[d]) return 0;
    return 1;
}

static int in_box(const int64_t *lo, const int64_t *hi, const int64_t *e)
{
    for (int d = 0; d < 3; d++)
        if (e[d] < lo[d] || e[d] >= hi[d]) return 0;
    return 1;
}

/* Offset clause composed with a work box W (Sec. 3, "Offset clauses"): element e of an array
 * of extent n is used (defined) by the work of W when some work item w in W touches e = w + o for
 * one of the offsets o.  A '*' component means the work item touches every element of that
 * dimension.  Elements outside the array are never touched (offsets that leave it are clipped). */
static int in_offsets(const int64_t *n, const int64_t *wlo, const int64_t *whi, int noff,
                      const int32_t *offs, const int64_t *e)
{
    if (!in_bounds(n, e)) return 0;
    for (int d = 0; d < 3; d++)
        if (whi[d] <= wlo[d]) return 0; /* empty work region touches nothing */
    for (int k = 0; k < noff; k++) {
        const int32_t *o = offs + 3 * k;
        int ok = 1;
        for (int d = 0; d < 3 && ok; d++) {
            if (o[d] == ORC_ALL) continue; /* some work item exists along d: W is not empty */
            int64_t w = e[d] - (int64_t)o[d];
            if (w < wlo[d] || w >= whi[d]) ok = 0;
        }
        if (ok) return 1;
    }
    return 0;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}

/* Trapezoid given by four corner elements (Sec. 3.1, HDArraySetTrapezoidUse/Def): upper-left,
 * upper-right, lower-left, lower-right, each (row, column).  Reading used here: the top edge is
 * the row of UL (= row of UR), the bottom edge the row of LL (= row of LR); in row r the element
 * columns run from the left edge to the right edge inclusive, each edge the straight line between
 * its two corners, rounded down (toward minus infinity) in exact integer arithmetic.
 * c = {ul_r, ul_c, ur_r, ur_c, ll_r, ll_c, lr_r, lr_c}. */
static int in_trapezoid(const int64_t *c, const int64_t *e)
{
    int64_t top = c[0], bottom = c[4];
    int64_t r = e[0], col = e[1];
    if (e[2] != 0) return 0;
    if (r < top || r > bottom) return 0;
    int64_t L, R;
    if (bottom == top) {
        L = c[1];
        R = c[3];
    } else {
        L = c[1] + floor_div((r - top) * (c[5] - c[1]), bottom - top);
        R = c[3] + floor_div((r - top) * (c[7] - c[3]), bottom - top);
    }
    return col >= L && col <= R;
}

static int trapezoid_valid(const int64_t *c)
{
    return c[0] == c[2] && c[4] == c[6] && c[0] <= c[4];
}

/* Mask builders: OR the predicate over every element of the array (row-major) into mask. */

static void coords_of(const int64_t *n, int64_t idx, int64_t *e)
{
    e[2] = idx % n[2];
    idx /= n[2];
    e[1] = idx % n[1];
    e[0] = idx / n[1];
}

void orc_mask_box(const int64_t *n, const int64_t *lo, const int64_t *hi, uint8_t *mask)
{
    int64_t total = n[0] * n[1] * n[2];
    int64_t e[3];
    for (int64_t i = 0; i < total; i++) {
        coords_of(n, i, e);
        if (in_box(lo, hi, e)) mask[i] = 1;
    }
}

void orc_mask_offsets(const int64_t *n, const int64_t *wlo, const int64_t *whi, int noff,
                      const int32_t *offs, uint8_t *mask)
{
    int64_t total = n[0] * n[1] * n[2];
    int64_t e[3];
    for (int64_t i = 0; i < total; i++) {
        coords_of(n, i, e);
        if (in_offsets(n, wlo, whi, noff, offs, e)) mask[i] = 1;
    }
}

int orc_mask_trapezoid(const int64_t *n, const int64_t *corners, uint8_t *mask)
{
    if (!trapezoid_valid(corners)) return -1;
    int64_t total = n[0] * n[1] * n[2];
    int64_t e[3];
    for (int64_t i = 0; i < total; i++) {
        coords_of(n, i, e);
        if (in_trapezoid(corners, e)) mask[i] = 1;
    }
    return 0;
}

/* The same predicates over an explicit list of elements (coords: 3 per element). */

void orc_pred_box(const int64_t *lo, const int64_t *hi, int64_t nel, const int64_t *coords,
                  uint8_t *out)
{
    for (int64_t i = 0; i < nel; i++)
        if (in_box(lo, hi, coords + 3 * i)) out[i] = 1;
}

void orc_pred_offsets(const int64_t *n, const int64_t *wlo, const int64_t *whi, int noff,
                      const int32_t *offs, int64_t nel, const int64_t *coords, uint8_t *out)
{
    for (int64_t i = 0; i < nel; i++)
        if (in_offsets(n, wlo, whi, noff, offs, coords + 3 * i)) out[i] = 1;
}

int orc_pred_trapezoid(const int64_t *corners, int64_t nel, const int64_t *coords, uint8_t *out)
{
    if (!trapezoid_valid(corners)) return -1;
    for (int64_t i = 0; i < nel; i++)
        if (in_trapezoid(corners, coords + 3 * i)) out[i] = 1;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Per-element state: who wrote each element last, and which devices hold its current value.   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int64_t total; /* number of tracked elements */
    int P;         /* number of devices */
    int16_t *owner; /* last writer, -1 while no device has written the element */
    uint8_t *have;  /* have[p * total + e]: device p holds the current value of e */
} orc_state;

/* A new HDArray: nothing has been written, so every device's (zeroed) copy is current and all
 * GDEF sets are empty (Sec. 2.1). */
orc_state *orc_state_new(int64_t total, int P)
{
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->total = total;
    s->P = P;
    s->owner = (int16_t *)malloc(sizeof(int16_t) * (size_t)(total > 0 ? total : 1));
    s->have = (uint8_t *)malloc((size_t)P * (size_t)(total > 0 ? total : 1));
    if (!s->owner || !s->have) {
        free(s->owner);
        free(s->have);
        free(s);
        return NULL;
    }
    for (int64_t e = 0; e < total; e++) s->owner[e] = -1;
    memset(s->have, 1, (size_t)P * (size_t)total);
    return s;
}

void orc_state_free(orc_state *s)
{
    if (!s) return;
    free(s->owner);
    free(s->have);
    free(s);
}

/* The message step of one call (Eq. 1 and 2).  use[p * total + e] marks LUSE_p.  For every device
 * p and every element it uses but does not hold, the last writer q = owner(e) sends e to p:
 * e is in sGDEF_{q,p} (q wrote it, has not sent it to p) and in LUSE_p.  Afterwards p holds e,
 * which removes e from sGDEF_{q,p} and rGDEF_{p,q} (the subtraction in Eq. 3 and 4).
 * src (optional, P * total): src[p * total + e] = q for a message q -> p, else -1.
 * counts (optional, P * P): counts[q * P + p] += number of elements sent from q to p.
 * Returns the number of messages, or -1 if an element is missing everywhere (cannot happen). */
int64_t orc_state_use(orc_state *s, const uint8_t *use, int16_t *src, int64_t *counts)
{
    int64_t T = s->total, nmsg = 0;
    int P = s->P;
    if (src)
        for (int64_t i = 0; i < (int64_t)P * T; i++) src[i] = -1;
    for (int p = 0; p < P; p++) {
        for (int64_t e = 0; e < T; e++) {
            if (!use[(int64_t)p * T + e]) continue;
            if (s->have[(int64_t)p * T + e]) continue;
            int q = s->owner[e];
            if (q < 0 || q >= P || !s->have[(int64_t)q * T + e]) return -1;
            if (src) src[(int64_t)p * T + e] = (int16_t)q;
            if (counts) counts[q * P + p] += 1;
            nmsg++;
        }
    }
    for (int p = 0; p < P; p++)
        for (int64_t e = 0; e < T; e++)
            if (use[(int64_t)p * T + e]) s->have[(int64_t)p * T + e] = 1;
    return nmsg;
}

/* The definition step of one call (Eq. 3 and 4, last writer wins).  def[p * total + e] marks
 * LDEF_p.  Two devices defining the same element in one call is a race (the paper assumes
 * race-free programs, Sec. 1): return -2 and change nothing.  Otherwise p becomes the owner of each
 * element it defines and every other device's copy of it becomes stale. */
int orc_state_def(orc_state *s, const uint8_t *def)
{
    int64_t T = s->total;
    int P = s->P;
    for (int64_t e = 0; e < T; e++) {
        int n = 0;
        for (int p = 0; p < P; p++) n += def[(int64_t)p * T + e] ? 1 : 0;
        if (n > 1) return -2;
    }
    for (int p = 0; p < P; p++) {
        for (int64_t e = 0; e < T; e++) {
            if (!def[(int64_t)p * T + e]) continue;
            s->owner[e] = (int16_t)p;
            for (int q = 0; q < P; q++) s->have[(int64_t)q * T + e] = (uint8_t)(q == p);
        }
    }
    return 0;
}

void orc_state_get(const orc_state *s, int16_t *owner, uint8_t *have)
{
    if (owner) memcpy(owner, s->owner, sizeof(int16_t) * (size_t)s->total);
    if (have) memcpy(have, s->have, (size_t)s->P * (size_t)s->total);
}

/* sGDEF_{p,q} as a mask: elements written by p that q does not hold (Sec. 2.1). */
void orc_state_sgdef(const orc_state *s, int p, int q, uint8_t *mask)
{
    for (int64_t e = 0; e < s->total; e++)
        mask[e] = (uint8_t)(p != q && s->owner[e] == p && !s->have[(int64_t)q * s->total + e]);
}

/* ------------------------------------------------------------------------------------------ */
/* Storage precisions.                                                                          */
/* ------------------------------------------------------------------------------------------ */

float orc_bf16_to_f32(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

/* binary32 -> bfloat16, round to nearest, ties to even (the 16 dropped bits decide; an exact tie
 * rounds to the even upper half).  NaN stays a quiet NaN of the same sign. */
uint16_t orc_f32_to_bf16(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0)
        return (uint16_t)((u >> 16) | 0x0040u);
    uint32_t upper = u >> 16;
    uint32_t lower = u & 0xffffu;
    if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1;
    return (uint16_t)upper;
}

void orc_f32_to_bf16_array(int64_t n, const float *in, uint16_t *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_f32_to_bf16(in[i]);
}

void orc_bf16_to_f32_array(int64_t n, const uint16_t *in, float *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = orc_bf16_to_f32(in[i]);
}

static double load_as_double(int prec, const void *X, int64_t i)
{
    if (prec == 0) return ((const double *)X)[i];
    if (prec == 1) return (double)((const float *)X)[i];
    return (double)orc_bf16_to_f32(((const uint16_t *)X)[i]);
}

/* ------------------------------------------------------------------------------------------ */
/* Workloads on the whole unpartitioned array.  Every call reads its inputs before any output is  */
/* written; input and output arrays are distinct.                                              */
/* ------------------------------------------------------------------------------------------ */

/* Jacobi step (Sec. 5): A[i][j] = (B[i][j-1] + B[i][j+1] + B[i-1][j] + B[i+1][j]) / 4,
 * summed left to right as printed, for every work element (work mask over the n0 x n1 array).
 * Returns -1 if a work element lacks a neighbour inside the array. */
int orc_jacobi2d(int prec, int64_t n0, int64_t n1, const void *B, void *A, const uint8_t *work)
{
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) num_threads(orc_nthreads)
    for (int64_t i = 0; i < n0; i++)
        for (int64_t j = 0; j < n1; j++)
            if (work[i * n1 + j] && (i == 0 || j == 0 || i == n0 - 1 || j == n1 - 1)) bad = 1;
    if (bad) return -1;
#pragma omp parallel for schedule(static) num_threads(orc_nthreads)
    for (int64_t i = 1; i < n0 - 1; i++) {
        for (int64_t j = 1; j + 1 < n1; j++) {
            int64_t c = i * n1 + j;
            if (!work[c]) continue;
            if (prec == 0) {
                const double *b = (const double *)B;
                double s = b[c - 1] + b[c + 1];
                s = s + b[c - n1];
                s = s + b[c + n1];
                ((double *)A)[c] = s / 4.0;
            } else if (prec == 1) {
                const float *b = (const float *)B;
                float s = b[c - 1] + b[c + 1];
                s = s + b[c - n1];
                s = s + b[c + n1];
                ((float *)A)[c] = s / 4.0f;
            } else {
                const uint16_t *b = (const uint16_t *)B;
                float s = orc_bf16_to_f32(b[c - 1]) + orc_bf16_to_f32(b[c + 1]);
                s = s + orc_bf16_to_f32(b[c - n1]);
                s = s + orc_bf16_to_f32(b[c + n1]);
                ((uint16_t *)A)[c] = orc_f32_to_bf16(s / 4.0f);
            }
        }
    }
    return 0;
}

/* 2-D convolution (Sec. 5: the Jacobi pattern plus the four diagonal neighbours, no dependency
 * between iterations).  The paper prints no coefficients, so the nine weights are arguments:
 *   A[i][j] = sum over a, b in 0..2 of w[3a + b] * B[i+a-1][j+b-1],
 * accumulated in that order starting from the first product, every product and sum rounded to
 * the arithmetic precision (binary64, or binary32 for float and bfloat16 storage, the weights
 * rounded to it first; bfloat16 results rounded to nearest even on the store).
 * Returns -1 if a work element lacks a neighbour inside the array. */
int orc_conv2d(int prec, int64_t n0, int64_t n1, const void *B, void *A, const uint8_t *work, const double *w)
{
    for (int64_t i = 0; i < n0; i++)
        for (int64_t j = 0; j < n1; j++)
            if (work[i * n1 + j] && (i == 0 || j == 0 || i == n0 - 1 || j == n1 - 1)) return -1;
    float wf[9];
    for (int k = 0; k < 9; k++) wf[k] = (float)w[k];
    for (int64_t i = 1; i + 1 < n0; i++) {
        for (int64_t j = 1; j + 1 < n1; j++) {
            const int64_t c = i * n1 + j;
            if (!work[c]) continue;
            if (prec == 0) {
                const double *b = (const double *)B;
                double s = w[0] * b[c - n1 - 1];
                for (int k = 1; k < 9; k++) s = s + w[k] * b[c + (k / 3 - 1) * n1 + (k % 3 - 1)];
                ((double *)A)[c] = s;
            } else if (prec == 1) {
                const float *b = (const float *)B;
                float s = wf[0] * b[c - n1 - 1];
                for (int k = 1; k < 9; k++) s = s + wf[k] * b[c + (k / 3 - 1) * n1 + (k % 3 - 1)];
                ((float *)A)[c] = s;
            } else {
                const uint16_t *b = (const uint16_t *)B;
                float s = wf[0] * orc_bf16_to_f32(b[c - n1 - 1]);
                for (int k = 1; k < 9; k++) s = s + wf[k] * orc_bf16_to_f32(b[c + (k / 3 - 1) * n1 + (k % 3 - 1)]);
                ((uint16_t *)A)[c] = orc_f32_to_bf16(s);
            }
        }
    }
    return 0;
}

/* 3-D 7-point analogue of the Jacobi step: the mean of the six face neighbours,
 * summed in the order x-1, x+1, y-1, y+1, z-1, z+1 (x = dimension 2, innermost; z = dimension 0),
 * then divided by 6 with one correctly rounded division. */
int orc_stencil3d(int prec, int64_t n0, int64_t n1, int64_t n2, const void *B, void *A,
                  const uint8_t *work)
{
    int64_t sz = n2, sy = n1 * n2;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) num_threads(orc_nthreads)
    for (int64_t z = 0; z < n0; z++)
        for (int64_t y = 0; y < n1; y++)
            for (int64_t x = 0; x < n2; x++)
                if (work[z * sy + y * sz + x] &&
                    (z == 0 || y == 0 || x == 0 || z == n0 - 1 || y == n1 - 1 || x == n2 - 1))
                    bad = 1;
    if (bad) return -1;
#pragma omp parallel for schedule(static) num_threads(orc_nthreads)
    for (int64_t z = 1; z < n0 - 1; z++) {
        for (int64_t y = 1; y + 1 < n1; y++) {
            for (int64_t x = 1; x + 1 < n2; x++) {
                int64_t c = z * sy + y * sz + x;
                if (!work[c]) continue;
                if (prec == 0) {
                    const double *b = (const double *)B;
                    double s = b[c - 1] + b[c + 1];
                    s = s + b[c - sz];
                    s = s + b[c + sz];
                    s = s + b[c - sy];
                    s = s + b[c + sy];
                    ((double *)A)[c] = s / 6.0;
                } else if (prec == 1) {
                    const float *b = (const float *)B;
                    float s = b[c - 1] + b[c + 1];
                    s = s + b[c - sz];
                    s = s + b[c + sz];
                    s = s + b[c - sy];
                    s = s + b[c + sy];
                    ((float *)A)[c] = s / 6.0f;
                } else {
                    const uint16_t *b = (const uint16_t *)B;
                    float s = orc_bf16_to_f32(b[c - 1]) + orc_bf16_to_f32(b[c + 1]);
                    s = s + orc_bf16_to_f32(b[c - sz]);
                    s = s + orc_bf16_to_f32(b[c + sz]);
                    s = s + orc_bf16_to_f32(b[c - sy]);
                    s = s + orc_bf16_to_f32(b[c + sy]);
                    ((uint16_t *)A)[c] = orc_f32_to_bf16(s / 6.0f);
                }
            }
        }
    }
    return 0;
}

/* Element copy Y = X over the work elements (the second Jacobi kernel of Sec. 5, B = A). */
void orc_copy(int prec, int64_t total, const void *X, void *Y, const uint8_t *work)
{
    int64_t es = prec == 0 ? 8 : (prec == 1 ? 4 : 2);
    for (int64_t i = 0; i < total; i++)
        if (work[i]) memcpy((char *)Y + i * es, (const char *)X + i * es, (size_t)es);
}

/* R = (X - Y)^2 in binary64 over the work elements (a residual field for HDArrayReduce). */
void orc_sqdiff(int prec, int64_t total, const void *X, const void *Y, double *R,
                const uint8_t *work)
{
    for (int64_t i = 0; i < total; i++) {
        if (!work[i]) continue;
        double d = load_as_double(prec, X, i) - load_as_double(prec, Y, i);
        R[i] = d * d;
    }
}

/* GEMM of Listing 3 in binary64: for every work element (i, j) of C,
 * C[i][j] *= beta; then for k = 0 .. nk-1: C[i][j] += alpha * A[i][k] * B[k][j]. */
void orc_gemm(int64_t ni, int64_t nj, int64_t nk, double alpha, double beta, const double *A,
              const double *B, double *C, const uint8_t *work)
{
    for (int64_t i = 0; i < ni; i++) {
        for (int64_t j = 0; j < nj; j++) {
            if (!work[i * nj + j]) continue;
            double c = C[i * nj + j] * beta;
            for (int64_t k = 0; k < nk; k++) c += alpha * A[i * nk + k] * B[k * nj + j];
            C[i * nj + j] = c;
        }
    }
}

/* The same GEMM for a list of (i, j) output entries only; out[t] receives the new C[i][j]. */
void orc_gemm_entries(int64_t nj, int64_t nk, double alpha, double beta, const double *A,
                      const double *B, const double *C, int64_t nent, const int64_t *ij,
                      double *out)
{
    for (int64_t t = 0; t < nent; t++) {
        int64_t i = ij[2 * t], j = ij[2 * t + 1];
        double c = C ? C[i * nj + j] * beta : 0.0;
        for (int64_t k = 0; k < nk; k++) c += alpha * A[i * nk + k] * B[k * nj + j];
        out[t] = c;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Covariance (Sec. 5.1: a triangular product, then a symmetric copy).  X is n x m: n samples of */
/* m variables.  binary64 or binary32 storage (prec 0 / 1).                                       */
/* ------------------------------------------------------------------------------------------ */

static void store_from_double(int prec, void *Y, int64_t i, double v)
{
    if (prec == 0) ((double *)Y)[i] = v;
    else ((float *)Y)[i] = (float)v;
}

/* Column means: M is 1 x m; for each work element (0, j): M[0][j] = (X[0][j] + ... + X[n-1][j]) / n,
 * summed in binary64 in row order, the quotient rounded to the storage type. */
int orc_colmean(int prec, int64_t n, int64_t m, const void *X, void *M, const uint8_t *work)
{
    if (prec > 1) return -1;
    for (int64_t j = 0; j < m; j++) {
        if (!work[j]) continue;
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) s += load_as_double(prec, X, i * m + j);
        store_from_double(prec, M, j, s / (double)n);
    }
    return 0;
}

/* Centring: for each work element (i, j): Xc[i][j] = X[i][j] - M[0][j], one subtraction in the
 * storage precision. */
int orc_center(int prec, int64_t n, int64_t m, const void *X, const void *M, void *Xc, const uint8_t *work)
{
    if (prec > 1) return -1;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < m; j++) {
            const int64_t c = i * m + j;
            if (!work[c]) continue;
            if (prec == 0) ((double *)Xc)[c] = ((const double *)X)[c] - ((const double *)M)[j];
            else ((float *)Xc)[c] = ((const float *)X)[c] - ((const float *)M)[j];
        }
    return 0;
}

/* Column norms (correlation): for each work element (0, j): S[0][j] = sqrt(sum_i X[i][j]^2), the
 * sum of squares in binary64 in row order, the root in binary64, rounded to the storage type. */
int orc_colnorm(int prec, int64_t n, int64_t m, const void *X, void *S, const uint8_t *work)
{
    if (prec > 1) return -1;
    for (int64_t j = 0; j < m; j++) {
        if (!work[j]) continue;
        double s = 0.0;
        for (int64_t i = 0; i < n; i++) {
            const double v = load_as_double(prec, X, i * m + j);
            s += v * v;
        }
        store_from_double(prec, S, j, sqrt(s));
    }
    return 0;
}

/* Column scaling (correlation): for each work element (i, j): Y[i][j] = X[i][j] / S[0][j], one
 * division in the storage precision. */
int orc_colscale(int prec, int64_t n, int64_t m, const void *X, const void *S, void *Y, const uint8_t *work)
{
    if (prec > 1) return -1;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < m; j++) {
            const int64_t c = i * m + j;
            if (!work[c]) continue;
            if (prec == 0) ((double *)Y)[c] = ((const double *)X)[c] / ((const double *)S)[j];
            else ((float *)Y)[c] = ((const float *)X)[c] / ((const float *)S)[j];
        }
    return 0;
}

/* Upper-triangular product: for each work element (i, j) of the m x m array C with j >= i:
 * C[i][j] = alpha * sum_k X[k][i] * X[k][j] (k ascending, binary64), rounded to the storage type.
 * Work elements with j < i are left alone. */
int orc_syrk_upper(int prec, int64_t n, int64_t m, double alpha, const void *X, void *C, const uint8_t *work)
{
    if (prec > 1) return -1;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = i; j < m; j++) {
            if (!work[i * m + j]) continue;
            double s = 0.0;
            for (int64_t k = 0; k < n; k++) s += load_as_double(prec, X, k * m + i) * load_as_double(prec, X, k * m + j);
            store_from_double(prec, C, i * m + j, alpha * s);
        }
    return 0;
}

/* Symmetric copy: for each work element (i, j) with j < i: C[i][j] = C[j][i] (a bit copy); work
 * elements with j >= i are left alone. */
int orc_symmetrize(int prec, int64_t m, void *C, const uint8_t *work)
{
    const int64_t es = prec == 0 ? 8 : prec == 1 ? 4 : 2;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < i; j++)
            if (work[i * m + j]) memcpy((char *)C + (i * m + j) * es, (const char *)C + (j * m + i) * es, (size_t)es);
    return 0;
}

/* HDArrayReduce (Table 2): fold the masked elements, in row-major order, in binary64.
 * op: 0 SUM, 1 PROD, 2 MAX, 3 MIN.  Returns -1 for an unknown op. */
int orc_reduce(int prec, int64_t total, const void *X, const uint8_t *mask, int op, double *out)
{
    double acc;
    if (op == 0) acc = 0.0;
    else if (op == 1) acc = 1.0;
    else if (op == 2) acc = -INFINITY;
    else if (op == 3) acc = INFINITY;
    else return -1;
    for (int64_t i = 0; i < total; i++) {
        if (!mask[i]) continue;
        double x = load_as_double(prec, X, i);
        if (op == 0) acc = acc + x;
        else if (op == 1) acc = acc * x;
        else if (op == 2) acc = x > acc ? x : acc;
        else acc = x < acc ? x : acc;
    }
    *out = acc;
    return 0;
}
