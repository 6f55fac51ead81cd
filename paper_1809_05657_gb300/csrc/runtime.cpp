// runtime.cpp -- the HDArray runtime on one GB300: arrays split over logical devices, section
// bookkeeping (Sec. 2), communication generation (Eq. 1-4), the call cache (Sec. 4.2), and the
// C ABI declared in include/hdarray.h.
#include "runtime.h"

#include <cudaTypedefs.h>

#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "hdarray.h"

using namespace hda;

namespace {

// ------------------------------------------------------------------------------------------
// Context
// ------------------------------------------------------------------------------------------

struct GraphRec {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    struct ArrInfo {
        HDArray *a;
        uint64_t generation, epoch;
        int pre, post;
    };
    std::vector<ArrInfo> arrays;
    std::vector<std::shared_ptr<Plan>> refs;
    std::vector<std::shared_ptr<DevMem>> mems;
    std::vector<HDArray *> defined;  // arrays the recorded calls define (their versions move on)
    int64_t nkernels = 0;
};

struct Ctx {
    bool inited = false;
    bool host_only = false;
    int ndev = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // asynchronous Write from host memory
    bool async_write = true;             // HDARRAY_ASYNC_WRITE=0: every Write on the library stream
    int mode = HDARRAY_MODE_FUSED;
    int nsm = 148;
    std::map<std::string, KernelDef> kernels;
    std::vector<Part> parts;
    std::set<HDArray *> arrays;
    uint64_t next_uid = 1, next_plan = 1;
    struct AbsSpec {
        std::map<int, std::vector<Box>> use, def;
        bool has_use = false, has_def = false;
        uint64_t version = 0;
    };
    std::map<std::tuple<std::string, int, uint64_t>, AbsSpec> abs;
    uint64_t abs_version = 1;
    std::unordered_map<std::string, std::shared_ptr<Plan>> memo;
    // batching
    bool batching = false;
    std::vector<std::shared_ptr<Plan>> batch;
    std::set<HDArray *> batch_used, batch_defined;  // arrays touched since HDArrayBatchBegin
    std::unordered_map<std::string, std::pair<std::shared_ptr<DevMem>, std::vector<LaunchRec>>> batch_cache;
    // graph recording
    bool recording = false, rec_invalid = false;
    std::vector<LaunchRec> rec;
    std::vector<std::shared_ptr<Plan>> rec_refs;
    std::vector<std::shared_ptr<DevMem>> rec_mems;
    std::map<HDArray *, std::pair<int, uint64_t>> rec_pre;  // state id, generation at first touch
    std::set<HDArray *> rec_defined;                         // arrays the recorded calls define
    std::map<int, GraphRec> graphs;
    int next_graph = 1;
    // the sum of the last residual launch's values (HDArrayReduce(R, SUM) over the same boxes,
    // while R is unchanged, reads it instead of folding R again)
    struct SqSum {
        HDArray *R = nullptr;
        uint64_t version = 0;
        std::vector<Box> boxes;
        std::shared_ptr<Plan> pl;  // keeps the scratch alive
        const double *sum = nullptr;
    } sq_sum;
    // reduction task tables per (array, partition, buffer epoch)
    struct RedPlan {
        std::shared_ptr<DevMem> mem;
        int ntasks = 0, nblocks = 0;
    };
    std::map<std::tuple<uint64_t, int, uint64_t>, RedPlan> red_plans;
    // reduction scratch
    double *red_partials = nullptr;
    unsigned *red_counter = nullptr;
    double *red_result = nullptr;
    unsigned *err_word = nullptr;  // set by kernels whose bounded waits gave up
    double *host_result = nullptr;
    int red_blocks = 0;
    // tunables
    int tile_rows = 32;     // 2-D tile height (rows per warp)
    int warps_per_cta = 8;  // 2-D warps per CTA
    int variant = 0;        // 2-D kernel variant (0 registers, 1 cp.async ring, 2 flat, 3 packed streams,
                            // 4 adaptive, 5 rows staged by bulk tensor copies)
    int tile_z = 64;        // 3-D tile depth (planes per tile)
    int variant3 = 1;       // 3-D kernel variant (0 warp per row, 1 CTA per tile with a plane ring, 2 flat,
                            // 3 the CTA tiles with planes staged by bulk tensor copies)
    int band2 = 32;         // 2-D packed-stream variant: most 16-byte chunks per band
    unsigned spin_limit = GEMM_SPIN_LIMIT_DEFAULT;  // polls of a GEMM pipeline wait (HDARRAY_SPIN_LIMIT)
    int band3 = 32;         // 3-D CTA variant: most 16-byte chunks per band
    int cta3 = 256;         // 3-D CTA variant: threads per CTA (256 or 512)
    int fuse = 1;           // exchange inside the stencil launch (1) or as a copy launch before it (0)
    int snake = 1;          // alternate the tile order of X -> Y and Y -> X launches (L2 reuse)
    int late = 1;           // 2-D TMA tiles issue their first copies before their receive (HDARRAY_LATE_RECEIVE)
    int gemm_parts = 2;     // binary32 GEMM on tensor cores: 2 bf16 parts (bf16x3) or 3 (bf16x6)
    int row_align = 16;     // bytes: device buffer rows start and end on this boundary (16 .. 1024)
    // autotuner: chosen tile shapes per (kernel, dtype, partition shape)
    bool autotune = false;
    bool tuning = false;  // compile_plan is being called by the tuner
    struct Shape { int variant, rows, warps, tile_z, fuse, variant3, band3, cta3, band2; };
    std::map<std::string, Shape> tuned;
    bool tune_file_loaded = false;  // HDARRAY_TUNE_CACHE read into `tuned` (once per HDArrayInit)
    // logical devices on several ranks (empty map: every device is local)
    std::vector<int> rank_of_dev;
    int my_rank = 0;
    HDArrayTransport_t transport = nullptr;
    void *transport_user = nullptr;
    // counters
    int64_t counters[5] = {0, 0, 0, 0, 0};
    int last_error = 0;
};

Ctx *g = nullptr;

int set_err(int code)
{
    if (g) g->last_error = code;
    return code;
}

#define CUDA_TRY(expr)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            if (getenv("HDARRAY_TRACE"))                                                     \
                fprintf(stderr, "hdarray: %s failed: %s\n", #expr, cudaGetErrorString(e_));  \
            return HDARRAY_ERR_CUDA;                                                         \
        }                                                                                    \
    } while (0)

bool trace() { return getenv("HDARRAY_TRACE") != nullptr; }

// Is logical device p mapped to this rank?
bool is_local(int p) { return g->rank_of_dev.empty() || g->rank_of_dev[p] == g->my_rank; }
int rank_of(int p) { return g->rank_of_dev.empty() ? 0 : g->rank_of_dev[p]; }

#define CUDA_OK(x)                           \
    do {                                     \
        if ((x) != cudaSuccess) {            \
            cudaGetLastError();              \
            return HDARRAY_ERR_CUDA;         \
        }                                    \
    } while (0)

// Library-stream work on a's buffers waits for an asynchronous Write of a still in flight.
int join_write(HDArray *a)
{
    if (!a->write_pending) return HDARRAY_OK;
    CUDA_OK(cudaStreamWaitEvent(g->stream, a->write_ev, 0));
    a->write_pending = false;
    return HDARRAY_OK;
}

// The library stream's work on a so far: the next asynchronous Write of a waits for it.
int note_use(HDArray *a)
{
    if (!a->track_use || g->host_only) return HDARRAY_OK;
    CUDA_OK(cudaEventRecord(a->use_ev, g->stream));
    return HDARRAY_OK;
}

int dtype_of(const char *t, int *esize)
{
    if (!t) return -1;
    if (!strcmp(t, "double")) { *esize = 8; return DT_F64; }
    if (!strcmp(t, "float")) { *esize = 4; return DT_F32; }
    if (!strcmp(t, "bf16") || !strcmp(t, "bfloat16")) { *esize = 2; return DT_BF16; }
    return -1;
}

// ------------------------------------------------------------------------------------------
// Built-in kernel table
// ------------------------------------------------------------------------------------------

Offset off(int a, int b, int c) { return Offset{{a, b, c}}; }

void register_builtins(Ctx &c)
{
    auto add = [&](KernelDef k) { c.kernels[k.name] = k; };
    const int ALL = OFFSET_ALL;
    {   // Sec. 5, Jacobi kernel 1: use B at (0,-1) (0,+1) (-1,0) (+1,0), define A at (0,0)
        KernelDef k;
        k.name = "jacobi2d"; k.kind = K_JACOBI2D; k.narr = 2; k.space = 1;
        k.use = {{off(0, -1, 0), off(0, 1, 0), off(-1, 0, 0), off(1, 0, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // Sec. 5, Jacobi kernel 2: B = A with zero offsets
        KernelDef k;
        k.name = "copy"; k.kind = K_COPY; k.narr = 2; k.space = 1;
        k.use = {{off(0, 0, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // Sec. 5, 2-D convolution: use A at the eight neighbours and the centre, define B at (0,0);
        // scalars: the nine weights, row-major over the offsets (-1,-1) .. (1,1)
        KernelDef k;
        k.name = "conv2d"; k.kind = K_CONV2D; k.narr = 2; k.nscal_f = 9; k.space = 1;
        std::vector<Offset> u;
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) u.push_back(off(a, b, 0));
        k.use = {u, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // Sec. 5.1 covariance: column means M (1 x m) of X (n x m); a work item (0, j) uses column j
        KernelDef k;
        k.name = "colmean"; k.kind = K_COLMEAN; k.narr = 2; k.space = 1;
        k.use = {{off(ALL, 0, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // centring Xc = X - M, M broadcast down the columns; args X, M, Xc
        KernelDef k;
        k.name = "center"; k.kind = K_CENTER; k.narr = 3; k.space = 2;
        k.use = {{off(0, 0, 0)}, {off(ALL, 0, 0)}, {}};
        k.def = {{}, {}, {off(0, 0, 0)}};
        add(k);
    }
    {   // correlation: column norms S (1 x m) of X, and Y = X / S; args (X, S) and (X, S, Y)
        KernelDef k;
        k.name = "colnorm"; k.kind = K_COLNORM; k.narr = 2; k.space = 1;
        k.use = {{off(ALL, 0, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
        KernelDef q;
        q.name = "colscale"; q.kind = K_COLSCALE; q.narr = 3; q.space = 2;
        q.use = {{off(0, 0, 0)}, {off(ALL, 0, 0)}, {}};
        q.def = {{}, {}, {off(0, 0, 0)}};
        add(q);
    }
    {   // C[i][j] = alpha (X^T X)[i][j] for j >= i; args X, C, alpha.  The use of X (columns i and j
        // of every row) is no offset pattern: all of X unless narrowed with absolute sections; the
        // definition is normally narrowed to the upper trapezoid of each device's rows
        KernelDef k;
        k.name = "syrk"; k.kind = K_SYRK; k.narr = 2; k.nscal_f = 1; k.space = 1;
        k.use = {{off(ALL, ALL, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // C[i][j] = C[j][i] for j < i (the symmetric copy); the transposed use likewise all of C
        // unless narrowed, the definition normally the lower trapezoid
        KernelDef k;
        k.name = "symmetrize"; k.kind = K_SYMM; k.narr = 1; k.space = 0;
        k.use = {{off(ALL, ALL, 0)}};
        k.def = {{off(0, 0, 0)}};
        add(k);
    }
    {   // 3-D 7-point analogue of Jacobi kernel 1
        KernelDef k;
        k.name = "stencil3d"; k.kind = K_STENCIL3D; k.narr = 2; k.space = 1;
        k.use = {{off(0, 0, -1), off(0, 0, 1), off(0, -1, 0), off(0, 1, 0), off(-1, 0, 0), off(1, 0, 0)}, {}};
        k.def = {{}, {off(0, 0, 0)}};
        add(k);
    }
    {   // the communication step alone: bring each device's use sections of X up to date
        KernelDef k;
        k.name = "exchange"; k.kind = K_EXCHANGE; k.narr = 1; k.space = 0;
        k.use = {{off(0, 0, 0)}};
        k.def = {{}};
        add(k);
    }
    {   // residual field R = (X - Y)^2
        KernelDef k;
        k.name = "sqdiff"; k.kind = K_SQDIFF; k.narr = 3; k.space = 2;
        k.use = {{off(0, 0, 0)}, {off(0, 0, 0)}, {}};
        k.def = {{}, {}, {off(0, 0, 0)}};
        add(k);
    }
    {   // Listing 3: use(A,(0,*)) use(B,(*,0)) def(C,(0,0)); args A, B, C, alpha, beta, ni, nj, nk
        KernelDef k;
        k.name = "gemm"; k.kind = K_GEMM; k.narr = 3; k.nscal_f = 2; k.nscal_i = 3; k.space = 2;
        k.use = {{off(0, ALL, 0)}, {off(ALL, 0, 0)}, {}};
        k.def = {{}, {}, {off(0, 0, 0)}};
        add(k);
        k.name = "trmm"; k.kind = K_TRMM; k.nscal_i = 0;
        add(k);
    }
}

// ------------------------------------------------------------------------------------------
// Arrays: state interning and device buffers
// ------------------------------------------------------------------------------------------

uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

uint64_t hash_state(const GState &s)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t p = 0; p < s.own.size(); p++) {
        h = mix64(h, (uint64_t)set_volume(s.own[p]) * 31 + p);
        h = mix64(h, (uint64_t)set_volume(s.stale[p]) * 37 + p);
        for (const Box &b : s.own[p])
            for (int d = 0; d < 3; d++) h = mix64(h, (uint64_t)(b.lo[d] * 131 + b.hi[d]));
    }
    return h;
}

bool state_equal(const GState &a, const GState &b)
{
    if (a.hash != b.hash || a.own.size() != b.own.size()) return false;
    for (size_t p = 0; p < a.own.size(); p++) {
        if (!set_equal(a.own[p], b.own[p])) return false;
        if (!set_equal(a.stale[p], b.stale[p])) return false;
    }
    return true;
}

int intern(HDArray *a, GState s)
{
    s.hash = hash_state(s);
    for (size_t i = 0; i < a->states.size(); i++)
        if (state_equal(a->states[i], s)) return (int)i;
    if (a->states.size() >= 4096) {  // bound the table: keep only the current state
        GState cur = a->states[a->cur];
        a->states.clear();
        a->states.push_back(cur);
        a->cur = 0;
        a->generation++;
        if (state_equal(a->states[0], s)) return 0;
    }
    a->states.push_back(std::move(s));
    return (int)a->states.size() - 1;
}

// Grow the number of tracked devices: a new device holds nothing that has been written.
void grow_devices(HDArray *a, int P)
{
    if (P <= a->P) return;
    for (GState &s : a->states) {
        BoxSet written;
        for (const BoxSet &o : s.own) written = set_union(written, o);
        while ((int)s.own.size() < P) {
            s.own.push_back({});
            s.stale.push_back(written);
        }
        s.hash = hash_state(s);
    }
    a->buf.resize(P);
    a->P = P;
}

int64_t align_down(int64_t v, int64_t a) { return v >= 0 ? (v / a) * a : -(((-v) + a - 1) / a) * a; }
int64_t align_up(int64_t v, int64_t a) { return align_down(v + a - 1, a); }

// Element offset of coordinate e (user order) inside a device buffer.
int64_t elem_off(const DevBuf &b, const int64_t e[3])
{
    return (e[0] - b.alloc.lo[0]) * b.st[0] + (e[1] - b.alloc.lo[1]) * b.st[1] +
           (e[2] - b.alloc.lo[2]) * b.st[2];
}

void set_strides(const HDArray *a, DevBuf &b)
{
    const Box &x = b.alloc;
    int64_t ext[3];
    for (int d = 0; d < 3; d++) ext[d] = x.hi[d] - x.lo[d];
    b.st[0] = b.st[1] = b.st[2] = 0;
    if (a->dim == 1) {
        b.st[0] = 1;
    } else if (a->dim == 2) {
        b.st[1] = 1;
        b.st[0] = ext[1];
    } else {
        b.st[2] = 1;
        b.st[1] = ext[2];
        b.st[0] = ext[2] * ext[1];
    }
}

int copy_box_d2d(const HDArray *a, const DevBuf &src, const DevBuf &dst, const Box &bx);

// Make device p's buffer of a cover box `need` (coordinates), reallocating if necessary.
int ensure_buffer(HDArray *a, int p, const Box &need)
{
    if (need.empty() || g->host_only) return HDARRAY_OK;
    DevBuf &b = a->buf[p];
    if (b.ptr && box_contains(b.alloc, need)) return HDARRAY_OK;
    if (g->recording) g->rec_invalid = true;  // recorded launches would point at the old buffer
    Box nb = b.ptr ? box_hull(b.alloc, need) : need;
    // Innermost dimension: rows padded to whole row_align-byte units (16 bytes unless set), with
    // the origin at 1 (mod the unit) in array coordinates, the same for every buffer.  Coordinate 1
    // -- the first element after a one-element boundary ring -- and every unit after it then start
    // a 16-byte chunk, so a work region that starts right after the ring is chunk-aligned for
    // vector access, and two buffers always agree on which coordinates are vector-aligned.  The
    // smallest unit keeps the rows of a narrow partition dense: consecutive rows share DRAM
    // sectors instead of each row touching its own partly used 128-byte line.
    const int in = a->dim - 1;
    const int64_t al = std::max<int64_t>(1, g->row_align / a->esize);
    nb.lo[in] = align_down(nb.lo[in] - 1, al) + 1;
    nb.hi[in] = align_up(nb.hi[in] - 1, al) + 1;
    DevBuf nbuf;
    nbuf.alloc = nb;
    set_strides(a, nbuf);
    nbuf.bytes = (size_t)nb.volume() * a->esize;
    void *ptr = nullptr;
    {
        const int arc = dev_alloc(&ptr, nbuf.bytes);
        if (arc) return arc;
    }
    nbuf.ptr = (char *)ptr;
    CUDA_TRY(cudaMemsetAsync(nbuf.ptr, 0, nbuf.bytes, g->stream));
    if (b.ptr) {
        int rc = copy_box_d2d(a, b, nbuf, b.alloc);
        if (rc) return rc;
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        dev_free(b.ptr);
    }
    b = nbuf;
    a->epoch++;
    return HDARRAY_OK;
}

// 3-level view of a box: outer x mid rows of inner contiguous elements.
struct View3 {
    int64_t n_outer, n_mid, n_inner;
    int64_t s_outer, s_mid;  // element strides in the buffer
};

View3 view_of(const HDArray *a, const DevBuf &b, const Box &bx)
{
    View3 v;
    if (a->dim == 1) {
        v.n_outer = 1; v.n_mid = 1; v.n_inner = bx.hi[0] - bx.lo[0];
        v.s_outer = 0; v.s_mid = 0;
    } else if (a->dim == 2) {
        v.n_outer = 1; v.n_mid = bx.hi[0] - bx.lo[0]; v.n_inner = bx.hi[1] - bx.lo[1];
        v.s_outer = 0; v.s_mid = b.st[0];
    } else {
        v.n_outer = bx.hi[0] - bx.lo[0]; v.n_mid = bx.hi[1] - bx.lo[1]; v.n_inner = bx.hi[2] - bx.lo[2];
        v.s_outer = b.st[0]; v.s_mid = b.st[1];
    }
    return v;
}

int vec_for(std::initializer_list<int64_t> vals)
{
    for (int v : {16, 8, 4, 2}) {
        bool ok = true;
        for (int64_t x : vals) ok = ok && (x % v == 0);
        if (ok) return v;
    }
    return 1;
}

const int64_t TASK_BYTES = 64 * 1024;
const int64_t TASK_ROWS = 1024;  // narrow rows (one-element faces) are split by count, not bytes

// Append copy tasks moving box bx of array a from device buffer src to device buffer dst.
void copy_tasks(const HDArray *a, const DevBuf &src, const DevBuf &dst, const Box &bx,
                std::vector<CopyTask> &out)
{
    if (bx.empty()) return;
    View3 vs = view_of(a, src, bx), vd = view_of(a, dst, bx);
    const int64_t es = a->esize;
    CopyTask t;
    t.src = src.ptr + elem_off(src, bx.lo) * es;
    t.dst = dst.ptr + elem_off(dst, bx.lo) * es;
    t.s_outer = vs.s_outer * es;
    t.s_mid = vs.s_mid * es;
    t.d_outer = vd.s_outer * es;
    t.d_mid = vd.s_mid * es;
    t.n_mid = (int32_t)vs.n_mid;
    t.inner = (int32_t)(vs.n_inner * es);
    t.vec = vec_for({(int64_t)(uintptr_t)t.src, (int64_t)(uintptr_t)t.dst, t.s_outer, t.s_mid,
                     t.d_outer, t.d_mid, (int64_t)t.inner});
    if (t.vec < 2) t.vec = 2;
    t.pad = 0;
    const int64_t rows = vs.n_outer * vs.n_mid;
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(TASK_ROWS, TASK_BYTES / std::max<int64_t>(1, t.inner)));
    for (int64_t r = 0; r < rows; r += per) {
        t.row_begin = (int32_t)r;
        t.row_end = (int32_t)std::min(rows, r + per);
        out.push_back(t);
    }
}

int upload(const std::vector<std::pair<const void *, size_t>> &parts, std::shared_ptr<DevMem> &mem,
           std::vector<const char *> &addrs)
{
    size_t total = 0;
    std::vector<size_t> offs;
    for (auto &p : parts) {
        offs.push_back(total);
        total += (p.second + 255) / 256 * 256;
    }
    mem = std::make_shared<DevMem>();
    addrs.clear();
    if (total == 0) {
        for (size_t i = 0; i < parts.size(); i++) addrs.push_back(nullptr);
        return HDARRAY_OK;
    }
    {
        const int arc = dev_alloc(&mem->ptr, total);
        if (arc) {
            mem->ptr = nullptr;
            return arc;
        }
    }
    mem->bytes = total;
    std::vector<char> host(total, 0);
    for (size_t i = 0; i < parts.size(); i++)
        if (parts[i].second) memcpy(host.data() + offs[i], parts[i].first, parts[i].second);
    CUDA_TRY(cudaMemcpy(mem->ptr, host.data(), total, cudaMemcpyHostToDevice));
    for (size_t i = 0; i < parts.size(); i++) addrs.push_back((const char *)mem->ptr + offs[i]);
    return HDARRAY_OK;
}

int copy_box_d2d(const HDArray *a, const DevBuf &src, const DevBuf &dst, const Box &bx)
{
    std::vector<CopyTask> tasks;
    copy_tasks(a, src, dst, bx, tasks);
    if (tasks.empty()) return HDARRAY_OK;
    std::shared_ptr<DevMem> mem;
    std::vector<const char *> addr;
    int rc = upload({{tasks.data(), tasks.size() * sizeof(CopyTask)}}, mem, addr);
    if (rc) return rc;
    CUDA_TRY(launch_copy((const CopyTask *)addr[0], (int)tasks.size(), g->stream));
    g->counters[0]++;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return HDARRAY_OK;
}

// ------------------------------------------------------------------------------------------
// Communication generation (Eq. 1-4)
// ------------------------------------------------------------------------------------------

// The message step for one array: for every device p, the elements of LUSE_p it does not hold
// come from their last writers.  SEND_{q,p} = sGDEF_{q,p} n LUSE_p = own[q] n stale[p] n LUSE_p
// (Eq. 1); RECV_{p,q} = SEND_{q,p} (Eq. 2).  Afterwards p holds all of LUSE_p (the subtraction of
// Eq. 3-4).
// The cross-rank moves of an exchange as transport records (HDARRAY_RANK_RECORD int64 each), sorted
// by source rank, then destination rank, then the exchange's order: every rank derives the same list
// from its replicated bookkeeping.
void rank_records(const HDArray *a, const std::vector<Move> &moves, std::vector<int64_t> &out)
{
    out.clear();
    if (g->rank_of_dev.empty()) return;
    std::vector<size_t> idx;
    for (size_t i = 0; i < moves.size(); i++)
        if (rank_of(moves[i].src) != rank_of(moves[i].dst)) idx.push_back(i);
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
        const int sx = rank_of(moves[x].src), sy = rank_of(moves[y].src);
        if (sx != sy) return sx < sy;
        return rank_of(moves[x].dst) < rank_of(moves[y].dst);
    });
    for (size_t i : idx) {
        const Move &m = moves[i];
        out.push_back(m.src);
        out.push_back(m.dst);
        out.push_back(rank_of(m.src));
        out.push_back(rank_of(m.dst));
        for (int d = 0; d < 3; d++) out.push_back(d < a->dim ? m.box.lo[d] : 0);
        for (int d = 0; d < 3; d++) out.push_back(d < a->dim ? m.box.hi[d] : 1);
    }
}

// Hand an exchange's cross-rank moves to the transport (nothing to do without any).
int run_transport(HDArray *a, const std::vector<Move> &moves)
{
    std::vector<int64_t> recs;
    rank_records(a, moves, recs);
    if (recs.empty()) return HDARRAY_OK;
    if (g->recording) return HDARRAY_ERR_UNSUPPORTED;
    if (!g->transport) return HDARRAY_ERR_STATE;
    return g->transport(a, (int64_t)(recs.size() / HDARRAY_RANK_RECORD), recs.data(), (void *)g->stream,
                        g->transport_user);
}

int use_step(GState &s, const std::vector<BoxSet> &luse, std::vector<Move> &moves)
{
    const int P = (int)s.own.size();
    for (int p = 0; p < (int)luse.size() && p < P; p++) {
        if (luse[p].empty()) continue;
        BoxSet need = set_intersect(luse[p], s.stale[p]);
        if (need.empty()) continue;
        int64_t got = 0;
        for (int q = 0; q < P; q++) {
            if (q == p) continue;
            BoxSet m = set_intersect(s.own[q], need);
            for (const Box &b : m) {
                moves.push_back(Move{q, p, b});
                got += b.volume();
            }
        }
        if (got != set_volume(need)) return HDARRAY_ERR_STATE;  // an element nobody holds
        s.stale[p] = set_subtract(s.stale[p], luse[p]);
    }
    return HDARRAY_OK;
}

// The definition step (Eq. 3-4, last writer wins): device p becomes the writer of LDEF_p, every
// other device's copy of it becomes stale, and older writers stop owning it.
int def_step(GState &s, const std::vector<BoxSet> &ldef)
{
    const int P = (int)s.own.size();
    for (int p = 0; p < (int)ldef.size(); p++)
        for (int q = p + 1; q < (int)ldef.size(); q++)
            if (!ldef[p].empty() && !ldef[q].empty() && set_overlaps(ldef[p], ldef[q]))
                return HDARRAY_ERR_RACE;
    for (int p = 0; p < (int)ldef.size() && p < P; p++) {
        const BoxSet &d = ldef[p];
        if (d.empty()) continue;
        for (int r = 0; r < P; r++) {
            if (r == p) {
                s.own[r] = set_union(s.own[r], d);
                s.stale[r] = set_subtract(s.stale[r], d);
            } else {
                if (!s.own[r].empty()) s.own[r] = set_subtract(s.own[r], d);
                s.stale[r] = set_union(s.stale[r], d);
            }
        }
    }
    return HDARRAY_OK;
}

// ------------------------------------------------------------------------------------------
// Sections of a call (LUSE/LDEF, Sec. 3 offset clauses and absolute sections)
// ------------------------------------------------------------------------------------------

BoxSet clip_set(const std::vector<Box> &boxes, const HDArray *a)
{
    Box ext = make_box(0, 0, 0, a->n[0], a->n[1], a->n[2]);
    std::vector<Box> c;
    for (const Box &b : boxes) {
        Box x = box_intersect(b, ext);
        if (!x.empty()) c.push_back(x);
    }
    return set_from_boxes(c);
}

void clause_sets(const Part &pt, const HDArray *a, const std::vector<Offset> &offs,
                 const std::map<int, std::vector<Box>> *absolute, std::vector<BoxSet> &out)
{
    out.assign(pt.nparts, BoxSet{});
    if (absolute) {
        for (auto &kv : *absolute)
            if (kv.first >= 0 && kv.first < pt.nparts) out[kv.first] = clip_set(kv.second, a);
        return;
    }
    if (offs.empty()) return;
    for (int p = 0; p < pt.nparts; p++) {
        const Box &w = pt.box[p];
        if (w.empty()) continue;
        std::vector<Box> bs;
        for (const Offset &o : offs) bs.push_back(offset_box(w, o.o, a->n));
        out[p] = set_from_boxes(bs);
    }
}

std::string memo_key(const KernelDef &k, int part, const std::vector<HDArray *> &args,
                     const std::vector<uint64_t> &absv, const std::vector<double> &scal)
{
    std::string key = k.name;
    char buf[96];
    snprintf(buf, sizeof(buf), "|%llu|%d", (unsigned long long)k.version, part);
    key += buf;
    for (size_t i = 0; i < args.size(); i++) {
        snprintf(buf, sizeof(buf), "|%llu:%llu:%d:%llu", (unsigned long long)args[i]->uid,
                 (unsigned long long)args[i]->generation, args[i]->cur,
                 (unsigned long long)absv[i]);
        key += buf;
    }
    for (double v : scal) {  // scalars are compiled into the launches
        snprintf(buf, sizeof(buf), "|%.17g", v);
        key += buf;
    }
    return key;
}

// ------------------------------------------------------------------------------------------
// Compiling a plan into launches
// ------------------------------------------------------------------------------------------

std::string epoch_sig(const Plan &pl)
{
    std::string s;
    char buf[48];
    for (HDArray *a : pl.args) {
        snprintf(buf, sizeof(buf), "%llu,", (unsigned long long)a->epoch);
        s += buf;
    }
    return s;
}

// Tiles of the fused Jacobi kernel for one device.  Returns false if the device's incoming
// sections are not exactly the halo strips of its tiles (then the exchange runs as a separate
// copy launch).
// Receive segments of a 2-D tile: the parts of the incoming moves on its four face strips.
// With `corners` the row strips extend one column past each end (the diagonal neighbours of a
// 3 x 3 operation); a corner cell then lies in the strips of up to three tiles, each of which
// copies it (the same bits) before reading it.
void tile2d_segments(const HDArray *X, const DevBuf &bx, StenTile2D &t, const std::vector<Move> &recv,
                     Sten2DHost &h, int64_t &covered, bool corners = false)
{
    const int e = corners ? 1 : 0;
    const Box strips[4] = {
        make_box(t.r0 - 1, t.c0 - e, 0, t.r0, t.c1 + e, 1), make_box(t.r1, t.c0 - e, 0, t.r1 + 1, t.c1 + e, 1),
        make_box(t.r0, t.c0 - 1, 0, t.r1, t.c0, 1), make_box(t.r0, t.c1, 0, t.r1, t.c1 + 1, 1)};
    for (const Move &m : recv) {
        const DevBuf &src = X->buf[m.src];
        for (int s = 0; s < 4; s++) {
            Box I = box_intersect(m.box, strips[s]);
            if (I.empty()) continue;
            Seg sg;
            sg.src = src.ptr + elem_off(src, I.lo) * X->esize;
            sg.dst = bx.ptr + elem_off(bx, I.lo) * X->esize;
            if (s < 2) {  // a row run
                sg.n = (int32_t)(I.hi[1] - I.lo[1]);
                sg.ss = 1;
                sg.ds = 1;
            } else {      // a column run
                sg.n = (int32_t)(I.hi[0] - I.lo[0]);
                sg.ss = src.st[0];
                sg.ds = bx.st[0];
            }
            sg.m = 1;
            sg.sso = 0;
            sg.dso = 0;
            covered += I.volume();
            h.segs.push_back(sg);
            t.nseg++;
        }
    }
}

bool encode_row_map(const HDArray *X, const DevBuf &b, int box_w, int box_h, CUtensorMap *out);

// Shape of the TMA 2-D kernel's tiles on one device's work box W: bands of equal width of at most
// band_chunks 16-byte chunks whose staged rows (band + 2 halo chunks) hold at most 256 elements;
// G row groups of JACOBI2D_TMA_ROWS rows per stage, so that G * nch <= 256 and a stage (its SR
// rows and 2 halo rows) holds at most JACOBI2D_TMA_STAGE_MAX bytes.
struct Tma2DGeom {
    int64_t cb0, nb, nch, rw, G, SR;  // first band column, bands, chunks per band, staged row width,
                                      // row groups, rows per stage
    size_t stage;                     // bytes of a stage, padded to 128
};
Tma2DGeom tma2d_geometry(const HDArray *X, const DevBuf &bx, const Box &W, int band_chunks)
{
    Tma2DGeom q;
    const int VEC = 16 / X->esize, M = JACOBI2D_TMA_ROWS;
    q.cb0 = bx.alloc.lo[1] + align_down(W.lo[1] - bx.alloc.lo[1], VEC);
    const int64_t chunks = (W.hi[1] - q.cb0 + VEC - 1) / VEC;
    const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(band_chunks, 256 / VEC - 2));
    q.nb = (chunks + cap - 1) / cap;
    q.nch = (chunks + q.nb - 1) / q.nb;
    q.rw = q.nch + 2;
    q.G = std::max<int64_t>(1, std::min<int64_t>({JACOBI2D_TMA_THREADS / q.nch, (int64_t)(254 / M),
                                                  (JACOBI2D_TMA_STAGE_MAX / (16 * q.rw) - 2) / M}));
    q.SR = q.G * M;
    q.stage = ((size_t)(q.SR + 2) * (size_t)q.rw * 16 + 127) / 128 * 128;
    return q;
}

// Received elements a TMA tile keeps for patching its first stages: the most any tile of h
// receives, rounded up to whole passes of the CTA's threads and capped at JACOBI2D_TMA_RX_MAX (a
// tile with more receives before its copies); 0 when no tile receives.
int tma2d_rx_cap(const Sten2DHost &h)
{
    int64_t most = 0;
    for (const StenTile2D &t : h.tiles) {
        int64_t n = 0;
        for (int s = 0; s < t.nseg; s++) n += (int64_t)h.segs[t.seg0 + s].n * h.segs[t.seg0 + s].m;
        most = std::max(most, n);
    }
    if (most == 0) return 0;
    const int64_t T = JACOBI2D_TMA_THREADS;
    return (int)std::min<int64_t>(JACOBI2D_TMA_RX_MAX, (most + T - 1) / T * T);
}

// Tiles of the fused 2-D kernel for one device.  Warp variants (0, 1): column bands of 32 chunks
// x tile_rows rows, a warp each.  Packed-stream variant (3): the box's chunks cut into bands of
// equal width of at most band_chunks (<= 32); per band, tiles of ns streams x sl rows with
// ns = min(256 / nch, 340 / (nch + 2)) and sl about tile_rows, balanced over the band's rows.
// TMA variant (5): the bands and stages of tma2d_geometry; tiles of whole stages, about
// 8 * tile_rows rows; one tensor map per part.
bool jacobi_tiles(const HDArray *X, const HDArray *Y, int p, const Box &W, int part_index,
                  const std::vector<Move> &recv, bool want_segs, Sten2DHost &h, int variant = 1,
                  int band_chunks = 32, bool corners = false)
{
    const DevBuf &bx = X->buf[p], &by = Y->buf[p];
    StenPart2D P{};
    P.x = bx.ptr;
    P.y = by.ptr;
    P.xlo0 = bx.alloc.lo[0];
    P.xlo1 = bx.alloc.lo[1];
    P.xs = bx.st[0];
    P.ylo0 = by.alloc.lo[0];
    P.ylo1 = by.alloc.lo[1];
    P.ys = by.st[0];
    h.parts.push_back(P);
    const int VEC = 16 / X->esize;
    const int H = std::max(1, g->tile_rows);
    bool exact = true;
    int64_t covered = 0, need = 0;
    for (const Move &m : recv) {
        need += m.box.volume();
        if (box_overlaps(m.box, W)) exact = false;
    }
    // bands start on 16-byte chunks of X's buffer (Y's buffer has the same phase, checked by the caller)
    const int64_t cb0 = bx.alloc.lo[1] + align_down(W.lo[1] - bx.alloc.lo[1], VEC);
    auto add = [&](StenTile2D &t) {
        t.part = part_index;
        t.seg0 = (int32_t)h.segs.size();
        t.nseg = 0;
        if (want_segs && exact) tile2d_segments(X, bx, t, recv, h, covered, corners);
        h.tiles.push_back(t);
    };
    // with corners every move outside W lies in the 1-ring of W, which the tiles' strips cover
    // (some cells more than once), so the fused form is exact iff no move reaches into W
    auto result = [&]() { return exact && (corners || covered == need); };
    if (variant == 5) {
        const Tma2DGeom q = tma2d_geometry(X, bx, W, band_chunks);
        const int64_t nb = q.nb, nch = q.nch, rw = q.rw, G = q.G, SR = q.SR;
        // tiles of whole stages, about 8 * tile_rows rows (only a band's last tile ends in a partial stage)
        const int64_t spt = std::max<int64_t>(1, (8 * (int64_t)H + SR / 2) / SR);
        const int64_t hr = spt * SR;
        h.smem = std::max(h.smem, (size_t)JACOBI2D_TMA_STAGES * q.stage + 128);
        h.parts.back().rwb = (int32_t)rw;
        CUtensorMap m;
        // a box's x coordinate (cb - VEC, from the buffer's first column) lies on a 16-byte boundary
        if ((cb0 - VEC - bx.alloc.lo[1]) % VEC != 0 || !encode_row_map(X, bx, (int)(rw * VEC), (int)(SR + 2), &m))
            h.map_error = true;
        h.maps.push_back(m);
        for (int64_t rb = W.lo[0]; rb < W.hi[0]; rb += hr) {
            for (int64_t b = 0; b < nb; b++) {
                const int64_t cb = cb0 + b * nch * VEC;
                StenTile2D t;
                t.r0 = (int32_t)rb;
                t.r1 = (int32_t)std::min<int64_t>(rb + hr, W.hi[0]);
                t.c0 = (int32_t)std::max<int64_t>(W.lo[1], cb);
                t.c1 = (int32_t)std::min<int64_t>(W.hi[1], cb + nch * VEC);
                t.cb = (int32_t)cb;
                t.nch = (int32_t)((t.c1 - cb + VEC - 1) / VEC);
                t.ns = (int32_t)G;
                t.sl = JACOBI2D_TMA_ROWS;
                add(t);
            }
        }
        return result();
    }
    if (variant == 3) {
        const int64_t chunks = (W.hi[1] - cb0 + VEC - 1) / VEC;
        const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(band_chunks, 32));
        const int64_t nb = (chunks + cap - 1) / cap;
        const int64_t nch = (chunks + nb - 1) / nb;
        // at most 340 staged slots (43.5 KB of ring per CTA): four CTAs per SM, the register limit
        const int64_t G = std::max<int64_t>(1, std::min<int64_t>(256 / nch, 340 / (nch + 2)));
        const int64_t R = W.hi[0] - W.lo[0];
        const int64_t ntr = (R + G * H - 1) / (G * H);     // tiles down the band
        const int64_t sl = (R + ntr * G - 1) / (ntr * G);  // balanced stream length
        h.smem = std::max(h.smem, (size_t)JACOBI2D_STAGES * G * (nch + 2) * 16);
        for (int64_t rb = W.lo[0]; rb < W.hi[0]; rb += G * sl) {
            for (int64_t b = 0; b < nb; b++) {
                const int64_t cb = cb0 + b * nch * VEC;
                StenTile2D t;
                t.r0 = (int32_t)rb;
                t.r1 = (int32_t)std::min<int64_t>(rb + G * sl, W.hi[0]);
                t.c0 = (int32_t)std::max<int64_t>(W.lo[1], cb);
                t.c1 = (int32_t)std::min<int64_t>(W.hi[1], cb + nch * VEC);
                t.cb = (int32_t)cb;
                t.nch = (int32_t)((t.c1 - cb + VEC - 1) / VEC);
                t.sl = (int32_t)sl;
                t.ns = (int32_t)((t.r1 - t.r0 + sl - 1) / sl);  // every stream has rows
                add(t);
            }
        }
        return result();
    }
    const int BAND = 32 * VEC;
    for (int64_t rb = W.lo[0]; rb < W.hi[0]; rb += H) {
        for (int64_t cb = cb0; cb < W.hi[1]; cb += BAND) {
            StenTile2D t;
            t.r0 = (int32_t)rb;
            t.r1 = (int32_t)std::min<int64_t>(rb + H, W.hi[0]);
            t.c0 = (int32_t)std::max<int64_t>(W.lo[1], cb);
            t.c1 = (int32_t)std::min<int64_t>(W.hi[1], cb + BAND);
            t.cb = (int32_t)cb;
            t.nch = 32;
            t.ns = 1;
            t.sl = t.r1 - t.r0;
            add(t);
        }
    }
    return result();
}

void box_segments(const HDArray *a, const DevBuf &src, const DevBuf &dst, const Box &I, std::vector<Seg> &out);

// Flat-block tiles of one device's work box (2-D): blocks up to 256 columns wide and about
// `cells` cells; the receive segments are the incoming cells on each block's four face strips.
bool flat2d_tiles(const HDArray *X, const HDArray *Y, int p, const Box &W, int part_index,
                  const std::vector<Move> &recv, bool want_segs, int cells, Sten2DHost &h)
{
    const DevBuf &bx = X->buf[p], &by = Y->buf[p];
    StenPart2D P{};
    P.x = bx.ptr; P.y = by.ptr;
    P.xlo0 = bx.alloc.lo[0]; P.xlo1 = bx.alloc.lo[1]; P.xs = bx.st[0];
    P.ylo0 = by.alloc.lo[0]; P.ylo1 = by.alloc.lo[1]; P.ys = by.st[0];
    h.parts.push_back(P);
    bool exact = true;
    int64_t covered = 0, need = 0;
    for (const Move &m : recv) {
        need += m.box.volume();
        if (box_overlaps(m.box, W)) exact = false;
    }
    const int64_t width = W.hi[1] - W.lo[1];
    const int64_t nbx = (width + 255) / 256;
    const int64_t bw = (width + nbx - 1) / nbx;  // balanced block widths
    const int64_t br = std::max<int64_t>(1, std::min<int64_t>(W.hi[0] - W.lo[0], cells / std::max<int64_t>(1, bw)));
    for (int64_t r = W.lo[0]; r < W.hi[0]; r += br) {
        for (int64_t c = W.lo[1]; c < W.hi[1]; c += bw) {
            StenTile2D t;
            t.nch = 0; t.ns = 0; t.sl = 0;
            t.part = part_index;
            t.r0 = (int32_t)r;
            t.r1 = (int32_t)std::min<int64_t>(r + br, W.hi[0]);
            t.c0 = (int32_t)c;
            t.c1 = (int32_t)std::min<int64_t>(c + bw, W.hi[1]);
            t.cb = t.c0;
            t.seg0 = (int32_t)h.segs.size();
            t.nseg = 0;
            if (want_segs && exact) {
                const Box strips[4] = {
                    make_box(t.r0 - 1, t.c0, 0, t.r0, t.c1, 1), make_box(t.r1, t.c0, 0, t.r1 + 1, t.c1, 1),
                    make_box(t.r0, t.c0 - 1, 0, t.r1, t.c0, 1), make_box(t.r0, t.c1, 0, t.r1, t.c1 + 1, 1)};
                for (const Move &m : recv)
                    for (int s = 0; s < 4; s++) {
                        Box I = box_intersect(m.box, strips[s]);
                        if (I.empty()) continue;
                        const size_t before = h.segs.size();
                        box_segments(X, X->buf[m.src], bx, I, h.segs);
                        t.nseg += (int32_t)(h.segs.size() - before);
                        covered += I.volume();
                    }
            }
            h.smem = std::max(h.smem, flat2d_smem(X->dtype, t.r1 - t.r0, t.c1 - t.c0));
            h.tiles.push_back(t);
        }
    }
    return exact && covered == need;
}

// A receive segment for box I (at most two dimensions longer than one element) moved from buffer
// src to buffer dst: the innermost long dimension is the inner run, the next one the outer run.
void box_segments(const HDArray *a, const DevBuf &src, const DevBuf &dst, const Box &I, std::vector<Seg> &out)
{
    int dims[3], nd = 0;
    for (int d = 2; d >= 0; d--)
        if (I.hi[d] - I.lo[d] > 1) dims[nd++] = d;
    if (nd == 3) {  // not a face: one segment per outermost index
        for (int64_t z = I.lo[0]; z < I.hi[0]; z++) {
            Box J = I;
            J.lo[0] = z;
            J.hi[0] = z + 1;
            box_segments(a, src, dst, J, out);
        }
        return;
    }
    Seg sg;
    sg.src = src.ptr + elem_off(src, I.lo) * a->esize;
    sg.dst = dst.ptr + elem_off(dst, I.lo) * a->esize;
    sg.n = 1; sg.ss = 1; sg.ds = 1;
    sg.m = 1; sg.sso = 0; sg.dso = 0;
    if (nd >= 1) {
        sg.n = (int32_t)(I.hi[dims[0]] - I.lo[dims[0]]);
        sg.ss = src.st[dims[0]];
        sg.ds = dst.st[dims[0]];
    }
    if (nd == 2) {
        sg.m = (int32_t)(I.hi[dims[1]] - I.lo[dims[1]]);
        sg.sso = src.st[dims[1]];
        sg.dso = dst.st[dims[1]];
    }
    out.push_back(sg);
}

// A tiled tensor map of `rank` dimensions (innermost first) over device buffer b of X, through the
// driver's encoder (found through the runtime; nothing links the driver library).  The checks are
// the encoder's documented rules: a 16-byte aligned base, strides in multiples of 16 bytes, boxes
// of 1 .. 256 elements per dimension with a whole number of 16-byte units in the inner one.
bool encode_tiled(const HDArray *X, const DevBuf &b, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
                  const cuuint32_t *box, CUtensorMap *out)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return false;
        }
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const CUtensorMapDataType dt = X->dtype == DT_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : X->dtype == DT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                        : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint32_t estr[3] = {1, 1, 1};
    if (((uintptr_t)b.ptr & 15) != 0 || (box[0] * X->esize) % 16 != 0) return false;
    for (int d = 0; d < rank; d++)
        if (box[d] < 1 || box[d] > 256 || dims[d] < 1) return false;
    for (int d = 0; d + 1 < rank; d++)
        if (strides[d] % 16 != 0) return false;
    return encode(out, dt, rank, b.ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D map of a 3-D array's buffer for boxes of box_w elements x box_h rows x one plane.
bool encode_box_map(const HDArray *X, const DevBuf &b, int box_w, int box_h, CUtensorMap *out)
{
    const cuuint64_t dims[3] = {(cuuint64_t)(b.alloc.hi[2] - b.alloc.lo[2]), (cuuint64_t)(b.alloc.hi[1] - b.alloc.lo[1]),
                                (cuuint64_t)(b.alloc.hi[0] - b.alloc.lo[0])};
    const cuuint64_t strides[2] = {(cuuint64_t)(b.st[1] * X->esize), (cuuint64_t)(b.st[0] * X->esize)};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    return encode_tiled(X, b, 3, dims, strides, box, out);
}

// 2-D map of a 2-D array's buffer for boxes of box_w elements x box_h rows.
bool encode_row_map(const HDArray *X, const DevBuf &b, int box_w, int box_h, CUtensorMap *out)
{
    const cuuint64_t dims[2] = {(cuuint64_t)(b.alloc.hi[1] - b.alloc.lo[1]), (cuuint64_t)(b.alloc.hi[0] - b.alloc.lo[0])};
    const cuuint64_t strides[1] = {(cuuint64_t)(b.st[0] * X->esize)};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    return encode_tiled(X, b, 2, dims, strides, box, out);
}

// Tiles of the fused 3-D kernel for one device, in (z chunk, x band, rows) order; the receive
// segments are the parts of the incoming faces on the tile's six face strips.  variant 0: bands
// of 32 chunks, one row per tile; variant 1: the box's chunks cut into bands of equal width of
// at most band_chunks, as many rows per tile as `threads` threads hold; variant 2 (flat_cells > 0):
// balanced widths up to 128 elements, rows so that a plane has about flat_cells cells.
bool stencil3d_tiles(const HDArray *X, const HDArray *Y, int p, const Box &W, int part_index,
                     const std::vector<Move> &recv, bool want_segs, int variant, Sten3DHost &h,
                     int flat_cells = 0, int band_chunks = 32, int threads = 256)
{
    const DevBuf &bx = X->buf[p], &by = Y->buf[p];
    StenPart3D P{};
    P.x = bx.ptr;
    P.y = by.ptr;
    P.xlo0 = bx.alloc.lo[0]; P.xlo1 = bx.alloc.lo[1]; P.xlo2 = bx.alloc.lo[2];
    P.xs0 = bx.st[0]; P.xs1 = bx.st[1];
    P.ylo0 = by.alloc.lo[0]; P.ylo1 = by.alloc.lo[1]; P.ylo2 = by.alloc.lo[2];
    P.ys0 = by.st[0]; P.ys1 = by.st[1];
    h.parts.push_back(P);
    const int VEC = 16 / X->esize;
    const int ZC = std::max(1, g->tile_z);
    bool exact = true;
    int64_t covered = 0, need = 0;
    for (const Move &m : recv) {
        need += m.box.volume();
        if (box_overlaps(m.box, W)) exact = false;
    }
    int64_t xb0 = bx.alloc.lo[2] + align_down(W.lo[2] - bx.alloc.lo[2], VEC);
    int64_t band = 32 * VEC;
    int rows_per_tile = 1;
    if (variant == 1) {
        // one chunk per thread; at most 2 * threads staged slots (two copy items per thread), and
        // at most 704 with 512 threads so that two CTAs' rings fit on an SM; a band of nch chunks
        // stages at least 3 (nch + 2) slots
        threads = threads == 512 ? 512 : 256;
        const int64_t slot_cap = threads == 512 ? 704 : 2 * threads;
        const int64_t chunks = (W.hi[2] - xb0 + VEC - 1) / VEC;
        const int64_t cap = std::max<int64_t>(1, std::min<int64_t>({(int64_t)band_chunks, (int64_t)threads, slot_cap / 3 - 2}));
        const int64_t nb = (chunks + cap - 1) / cap;
        const int64_t nch = (chunks + nb - 1) / nb;
        band = nch * VEC;
        rows_per_tile = (int)std::max<int64_t>(1, std::min<int64_t>(threads / nch, slot_cap / (nch + 2) - 2));
        h.smem = std::max(h.smem, (size_t)STENCIL3D_STAGES * (rows_per_tile + 2) * (nch + 2) * 16);
    } else if (variant == 3) {
        // the variant-1 tiles, planes staged by TMA: a box row of nch + 2 chunks holds at most 256
        // elements; stages padded to 128 bytes, plus 128 bytes to align the ring
        threads = threads == 512 ? 512 : 256;
        const int64_t slot_cap = threads == 512 ? 704 : 2 * threads;
        const int64_t chunks = (W.hi[2] - xb0 + VEC - 1) / VEC;
        const int64_t cap = std::max<int64_t>(1, std::min<int64_t>({(int64_t)band_chunks, (int64_t)threads,
                                                                    slot_cap / 3 - 2, (int64_t)(256 / VEC - 2)}));
        const int64_t nb = (chunks + cap - 1) / cap;
        const int64_t nch = (chunks + nb - 1) / nb;
        band = nch * VEC;
        rows_per_tile = (int)std::max<int64_t>(1, std::min<int64_t>(threads / nch, slot_cap / (nch + 2) - 2));
        const int64_t slots = ((rows_per_tile + 2) * (nch + 2) + 7) / 8 * 8;
        h.smem = std::max(h.smem, (size_t)STENCIL3D_STAGES * slots * 16 + 128);
        h.parts.back().rwb = (int32_t)(nch + 2);
        h.parts.back().boxh = (int32_t)(rows_per_tile + 2);
        CUtensorMap m;
        if (!encode_box_map(X, bx, (int)((nch + 2) * VEC), rows_per_tile + 2, &m)) h.map_error = true;
        h.maps.push_back(m);
    }
    if (flat_cells > 0) {
        const int64_t width = W.hi[2] - W.lo[2];
        const int64_t nbx = (width + 127) / 128;
        band = (width + nbx - 1) / nbx;
        xb0 = W.lo[2];
        rows_per_tile = (int)std::max<int64_t>(1, std::min<int64_t>(W.hi[1] - W.lo[1], flat_cells / band));
    }
    for (int64_t zc = W.lo[0]; zc < W.hi[0]; zc += ZC) {
        for (int64_t xb = xb0; xb < W.hi[2]; xb += band) {
            for (int64_t y = W.lo[1]; y < W.hi[1]; y += rows_per_tile) {
                StenTile3D t;
                t.part = part_index;
                t.z0 = (int32_t)zc;
                t.z1 = (int32_t)std::min<int64_t>(zc + ZC, W.hi[0]);
                t.y = (int32_t)y;
                t.ny = (int32_t)std::min<int64_t>(rows_per_tile, W.hi[1] - y);
                t.x0 = (int32_t)std::max<int64_t>(W.lo[2], xb);
                t.x1 = (int32_t)std::min<int64_t>(W.hi[2], xb + band);
                t.xb = (int32_t)xb;
                t.nch = (int32_t)((t.x1 - xb + VEC - 1) / VEC);
                t.seg0 = (int32_t)h.segs.size();
                t.nseg = 0;
                if (want_segs && exact) {
                    const int64_t y1 = y + t.ny;
                    const Box strips[6] = {
                        make_box(t.z0 - 1, y, t.x0, t.z0, y1, t.x1), make_box(t.z1, y, t.x0, t.z1 + 1, y1, t.x1),
                        make_box(t.z0, y - 1, t.x0, t.z1, y, t.x1), make_box(t.z0, y1, t.x0, t.z1, y1 + 1, t.x1),
                        make_box(t.z0, y, t.x0 - 1, t.z1, y1, t.x0), make_box(t.z0, y, t.x1, t.z1, y1, t.x1 + 1)};
                    for (const Move &m : recv) {
                        for (int s = 0; s < 6; s++) {
                            Box I = box_intersect(m.box, strips[s]);
                            if (I.empty()) continue;
                            const size_t before = h.segs.size();
                            box_segments(X, X->buf[m.src], bx, I, h.segs);
                            t.nseg += (int32_t)(h.segs.size() - before);
                            covered += I.volume();
                        }
                    }
                }
                if (flat_cells > 0) h.smem = std::max(h.smem, flat3d_smem(X->dtype, t.ny, t.x1 - t.x0));
                h.tiles.push_back(t);
            }
        }
    }
    return exact && covered == need;
}

int compile_plan(Plan &pl)
{
    pl.launches.clear();
    pl.user_work.clear();
    pl.copy_host.clear();
    pl.s2 = Sten2DHost{};
    pl.fused = false;
    pl.tables.reset();
    const KernelDef &k = *pl.k;
    // with devices on several ranks this rank compiles its own devices' work (the others' boxes
    // empty) and the moves between its own devices; cross-rank moves arrive through the transport
    Part local_part;
    if (!g->rank_of_dev.empty()) {
        local_part = g->parts[pl.part];
        for (int p = 0; p < local_part.nparts; p++)
            if (!is_local(p)) local_part.box[p] = Box{};
    }
    const Part &pt = g->rank_of_dev.empty() ? g->parts[pl.part] : local_part;
    auto local_move = [](const Move &m) { return is_local(m.src) && is_local(m.dst); };
    const bool plain = g->mode == HDARRAY_MODE_PLAIN;
    std::vector<std::pair<const void *, size_t>> blobs;

    // every exchange of every array, as copy tasks (one group per move for the plain form)
    std::vector<CopyTask> xfer;
    std::vector<std::pair<int, int>> xfer_groups;  // [begin, end) per move
    auto add_moves = [&](const ArrStep &st) {
        for (const Move &m : st.moves) {
            if (!local_move(m)) continue;
            int b = (int)xfer.size();
            copy_tasks(st.a, st.a->buf[m.src], st.a->buf[m.dst], m.box, xfer);
            xfer_groups.push_back({b, (int)xfer.size()});
        }
    };

    if (k.kind == K_JACOBI2D || k.kind == K_CONV2D) {
        const bool conv = k.kind == K_CONV2D;  // the packed-stream kernel, or rows staged by TMA
        HDArray *X = pl.args[0], *Y = pl.args[1];
        const ArrStep *sx = nullptr;
        for (const ArrStep &st : pl.steps)
            if (st.a == X) sx = &st;
        bool fused = !plain && g->fuse;
        Sten2DHost h;
        h.dtype = X->dtype;
        std::vector<std::pair<int, int>> dev_ranges;
        int idx = 0;
        const int VEC2 = 16 / X->esize;
        // variant 4 (adaptive): the packed-stream kernel when every part is narrower than half a
        // warp band (16 chunks), else the cp.async warp kernel
        int adaptive = 1;
        if (g->variant == 4) {
            int64_t widest = 0;
            for (int p = 0; p < pt.nparts; p++)
                if (!pt.box[p].empty()) widest = std::max<int64_t>(widest, (pt.box[p].hi[1] - pt.box[p].lo[1] + VEC2) / VEC2);
            adaptive = widest < 16 ? 3 : 1;
        }
        // the TMA variant falls back to the packed-stream tiles where a buffer admits no tensor map
        const bool fuse0 = fused;
        for (int attempt = 0; attempt < 2; attempt++) {
            const int want = attempt ? 3 : g->variant;
            h = Sten2DHost{};
            h.dtype = X->dtype;
            dev_ranges.clear();
            idx = 0;
            fused = fuse0;
            for (int p = 0; p < pt.nparts; p++) {
                if (pt.box[p].empty()) continue;
                if ((Y->buf[p].alloc.lo[1] - X->buf[p].alloc.lo[1]) % VEC2 != 0) return HDARRAY_ERR_STATE;
                std::vector<Move> recv;
                if (sx)
                    for (const Move &m : sx->moves)
                        if (m.dst == p && local_move(m)) recv.push_back(m);
                int t0 = (int)h.tiles.size();
                const bool flat = !conv && want == 2 && X->dtype != DT_BF16;
                h.flat = flat;
                h.variant = conv ? (want == 5 ? 5 : 3) : flat ? 2 : want == 2 ? 1 : want == 4 ? adaptive : want;
                h.warps = g->warps_per_cta;
                bool ok = flat ? flat2d_tiles(X, Y, p, pt.box[p], idx++, recv, fused, g->tile_rows * 256, h)
                               : jacobi_tiles(X, Y, p, pt.box[p], idx++, recv, fused, h, h.variant, g->band2, conv);
                if (!ok) fused = false;
                dev_ranges.push_back({t0, (int)h.tiles.size()});
            }
            if (!(h.variant == 5 && h.map_error)) break;
        }
        if (!fused) {  // drop the segments: the exchange runs as copies
            h.segs.clear();
            for (StenTile2D &t : h.tiles) { t.seg0 = 0; t.nseg = 0; }
            if (sx) add_moves(*sx);
        }
        if (h.variant == 5 && g->late) h.rx_cap = tma2d_rx_cap(h);
        // one launch for every device: the tiles of the calls X -> Y and Y -> X run in opposite
        // orders, so an iteration starts on the rows the previous one wrote last, still in L2
        if (!plain && g->snake && X->uid > Y->uid) std::reverse(h.tiles.begin(), h.tiles.end());
        blobs.push_back({xfer.data(), xfer.size() * sizeof(CopyTask)});
        blobs.push_back({h.parts.data(), h.parts.size() * sizeof(StenPart2D)});
        blobs.push_back({h.tiles.data(), h.tiles.size() * sizeof(StenTile2D)});
        blobs.push_back({h.segs.data(), h.segs.size() * sizeof(Seg)});
        double wts[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int i = 0; i < 9 && conv; i++) wts[i] = i < (int)pl.scal.size() ? pl.scal[i] : 0.0;
        blobs.push_back({wts, conv ? sizeof(wts) : 0});
        // the same tiles in the reverse order: a convolution repeated on the same input (no
        // dependency across iterations) runs every other call with them, starting on the rows the
        // previous call read last, and the autotuner times candidate shapes that way (a ping-pong's
        // calls X -> Y and Y -> X get opposite orders from the rule above)
        std::vector<StenTile2D> rtiles;
        const bool alternate = !plain && g->snake && !h.tiles.empty();
        if (alternate) rtiles.assign(h.tiles.rbegin(), h.tiles.rend());
        blobs.push_back({rtiles.data(), rtiles.size() * sizeof(StenTile2D)});
        blobs.push_back({h.maps.data(), h.maps.size() * sizeof(CUtensorMap)});  // 128 bytes each
        std::vector<const char *> addr;
        int rc = upload(blobs, pl.tables, addr);
        if (rc) return rc;
        const CopyTask *dx = (const CopyTask *)addr[0];
        const int kind2d = conv ? L_CONV2D : h.flat ? L_FLAT2D : L_JACOBI2D;
        const char *p3 = h.variant == 5 ? addr[6] : addr[4];  // tensor maps, or the convolution's weights
        const char *p4 = h.variant == 5 && conv ? addr[4] : nullptr;  // the weights beside the maps
        if (plain) {
            for (auto &gr : xfer_groups)
                if (gr.second > gr.first) {
                    LaunchRec L; L.kind = L_COPY; L.p0 = dx + gr.first; L.n0 = gr.second - gr.first;
                    pl.launches.push_back(L);
                }
            for (auto &r : dev_ranges) {
                if (r.second <= r.first) continue;
                LaunchRec L; L.kind = kind2d; L.dtype = X->dtype; L.p3 = p3; L.p4 = p4;
                L.p0 = addr[1]; L.p1 = (const StenTile2D *)addr[2] + r.first; L.p2 = addr[3];
                L.n0 = r.second - r.first; L.n1 = h.flat ? (int64_t)h.smem : h.variant == 5 ? h.rx_cap : h.warps;
                L.n2 = h.variant; L.n3 = (int64_t)h.smem;
                pl.launches.push_back(L);
            }
        } else {
            if (!xfer.empty()) {
                LaunchRec L; L.kind = L_COPY; L.p0 = dx; L.n0 = (int64_t)xfer.size();
                pl.launches.push_back(L);
            }
            if (!h.tiles.empty()) {
                LaunchRec L; L.kind = kind2d; L.dtype = X->dtype; L.p3 = p3; L.p4 = p4;
                L.p0 = addr[1]; L.p1 = addr[2]; L.p2 = addr[3];
                if (alternate) {
                    L.p1_alt = addr[5];
                    L.alt_calls = conv;
                }
                L.n0 = (int64_t)h.tiles.size(); L.n1 = h.flat ? (int64_t)h.smem : h.variant == 5 ? h.rx_cap : h.warps;
                L.n2 = h.variant; L.n3 = (int64_t)h.smem;
                pl.launches.push_back(L);
            }
        }
        pl.fused = fused;
        pl.copy_host = xfer;
        pl.s2 = std::move(h);
        return HDARRAY_OK;
    }

    if (k.kind == K_STENCIL3D) {
        HDArray *X = pl.args[0], *Y = pl.args[1];
        const ArrStep *sx = nullptr;
        for (const ArrStep &st : pl.steps)
            if (st.a == X) sx = &st;
        bool fused = !plain && g->fuse;
        Sten3DHost h;
        std::vector<std::pair<int, int>> dev_ranges;
        int idx = 0;
        const int VEC = 16 / X->esize;
        // the TMA variant falls back to the cp.async tiles where a buffer admits no tensor map
        const bool fuse0 = fused;
        int v3 = g->variant3;
        for (int attempt = 0; attempt < 2; attempt++) {
            h = Sten3DHost{};
            h.dtype = X->dtype;
            dev_ranges.clear();
            idx = 0;
            fused = fuse0;
            for (int p = 0; p < pt.nparts; p++) {
                if (pt.box[p].empty()) continue;
                if ((Y->buf[p].alloc.lo[2] - X->buf[p].alloc.lo[2]) % VEC != 0) return HDARRAY_ERR_STATE;
                std::vector<Move> recv;
                if (sx)
                    for (const Move &m : sx->moves)
                        if (m.dst == p && local_move(m)) recv.push_back(m);
                int t0 = (int)h.tiles.size();
                const bool flat = v3 == 2 && X->dtype != DT_BF16;
                h.flat = flat;
                if (!stencil3d_tiles(X, Y, p, pt.box[p], idx++, recv, fused, flat ? 2 : v3, h,
                                     flat ? g->tile_rows * 64 : 0, g->band3, g->cta3))
                    fused = false;
                dev_ranges.push_back({t0, (int)h.tiles.size()});
            }
            if (!(v3 == 3 && h.map_error)) break;
            v3 = 1;
        }
        if (!fused) {
            h.segs.clear();
            for (StenTile3D &t : h.tiles) { t.seg0 = 0; t.nseg = 0; }
            if (sx) add_moves(*sx);
        }
        if (!plain && g->snake && X->uid > Y->uid) std::reverse(h.tiles.begin(), h.tiles.end());
        blobs.push_back({xfer.data(), xfer.size() * sizeof(CopyTask)});
        blobs.push_back({h.parts.data(), h.parts.size() * sizeof(StenPart3D)});
        blobs.push_back({h.tiles.data(), h.tiles.size() * sizeof(StenTile3D)});
        blobs.push_back({h.segs.data(), h.segs.size() * sizeof(Seg)});
        std::vector<StenTile3D> rtiles;  // the same tiles reversed: the autotuner's alternating runs
        const bool alternate = !plain && g->snake && !h.tiles.empty();
        if (alternate) rtiles.assign(h.tiles.rbegin(), h.tiles.rend());
        blobs.push_back({rtiles.data(), rtiles.size() * sizeof(StenTile3D)});
        blobs.push_back({h.maps.data(), h.maps.size() * sizeof(CUtensorMap)});  // 128 bytes each
        std::vector<const char *> addr;
        int rc = upload(blobs, pl.tables, addr);
        if (rc) return rc;
        const CopyTask *dx = (const CopyTask *)addr[0];
        if (plain) {
            for (auto &gr : xfer_groups)
                if (gr.second > gr.first) {
                    LaunchRec L; L.kind = L_COPY; L.p0 = dx + gr.first; L.n0 = gr.second - gr.first;
                    pl.launches.push_back(L);
                }
            for (auto &r : dev_ranges) {
                if (r.second <= r.first) continue;
                LaunchRec L; L.kind = h.flat ? L_FLAT3D : L_STENCIL3D; L.dtype = X->dtype;
                L.p0 = addr[1]; L.p1 = (const StenTile3D *)addr[2] + r.first; L.p2 = addr[3]; L.p3 = addr[5];
                L.n0 = r.second - r.first; L.n1 = h.flat ? (int64_t)h.smem : g->cta3 / 32; L.n2 = v3; L.n3 = (int64_t)h.smem;
                pl.launches.push_back(L);
            }
        } else {
            if (!xfer.empty()) {
                LaunchRec L; L.kind = L_COPY; L.p0 = dx; L.n0 = (int64_t)xfer.size();
                pl.launches.push_back(L);
            }
            if (!h.tiles.empty()) {
                LaunchRec L; L.kind = h.flat ? L_FLAT3D : L_STENCIL3D; L.dtype = X->dtype;
                L.p0 = addr[1]; L.p1 = addr[2]; L.p2 = addr[3]; L.p3 = addr[5];
                if (alternate) L.p1_alt = addr[4];
                L.n0 = (int64_t)h.tiles.size(); L.n1 = h.flat ? (int64_t)h.smem : g->cta3 / 32; L.n2 = v3; L.n3 = (int64_t)h.smem;
                pl.launches.push_back(L);
            }
        }
        pl.fused = fused;
        pl.copy_host = xfer;
        pl.s3 = std::move(h);
        return HDARRAY_OK;
    }

    for (const ArrStep &st : pl.steps) add_moves(st);
    std::vector<CopyTask> local;       // within-device copies (kernel "copy")
    std::vector<std::pair<int, int>> local_groups;
    std::vector<PwTask> pw;
    std::vector<std::pair<int, int>> pw_groups;
    std::vector<GemmPart> gp;
    std::vector<TcPart> tp;
    std::vector<TcTile> tt;
    std::vector<CovTask> cov;
    int max_rows = 0, max_cols = 0;
    for (int p = 0; p < pt.nparts; p++) {
        const Box &W = pt.box[p];
        if (W.empty()) continue;
        if (k.kind == K_COPY) {
            int b = (int)local.size();
            copy_tasks(pl.args[0], pl.args[0]->buf[p], pl.args[1]->buf[p], W, local);
            local_groups.push_back({b, (int)local.size()});
        } else if (k.kind == K_SQDIFF) {
            HDArray *X = pl.args[0], *Y = pl.args[1], *R = pl.args[2];
            const DevBuf &bx = X->buf[p], &by = Y->buf[p], &br = R->buf[p];
            View3 vx = view_of(X, bx, W), vy = view_of(Y, by, W), vr = view_of(R, br, W);
            PwTask t;
            t.x = bx.ptr + elem_off(bx, W.lo) * X->esize;
            t.y = by.ptr + elem_off(by, W.lo) * Y->esize;
            t.r = (double *)(br.ptr + elem_off(br, W.lo) * 8);
            t.xs_outer = vx.s_outer; t.xs_mid = vx.s_mid;
            t.ys_outer = vy.s_outer; t.ys_mid = vy.s_mid;
            t.rs_outer = vr.s_outer; t.rs_mid = vr.s_mid;
            t.n_mid = (int32_t)vx.n_mid; t.n_inner = (int32_t)vx.n_inner;
            const int64_t rows = vx.n_outer * vx.n_mid;
            const int64_t per = std::max<int64_t>(1, 65536 / std::max<int64_t>(1, vx.n_inner));
            int b = (int)pw.size();
            for (int64_t r = 0; r < rows; r += per) {
                t.row_begin = (int32_t)r;
                t.row_end = (int32_t)std::min(rows, r + per);
                pw.push_back(t);
            }
            pw_groups.push_back({b, (int)pw.size()});
        } else if (k.kind == K_USER) {
            HDArrayWork_t w;
            memset(&w, 0, sizeof(w));
            w.dev = p;
            for (int d = 0; d < 3; d++) {
                w.lo[d] = W.lo[d];
                w.hi[d] = W.hi[d];
            }
            for (int i = 0; i < (int)pl.args.size() && i < HDARRAY_MAX_KERNEL_ARRAYS; i++) {
                const DevBuf &b = pl.args[i]->buf[p];
                w.buf[i] = b.ptr;
                for (int d = 0; d < 3; d++) {
                    w.buf_lo[i][d] = b.alloc.lo[d];
                    w.buf_stride[i][d] = b.st[d];
                }
            }
            pl.user_work.push_back(w);
        } else if (k.kind == K_COLMEAN || k.kind == K_CENTER || k.kind == K_SYMM || k.kind == K_COLNORM ||
                   k.kind == K_COLSCALE) {
            const bool reduce_cols = k.kind == K_COLMEAN || k.kind == K_COLNORM;
            const bool pointwise = k.kind == K_CENTER || k.kind == K_COLSCALE;
            HDArray *X = pl.args[0];
            const DevBuf &bx = X->buf[p];
            CovTask t;
            t.x = bx.ptr; t.m = nullptr; t.y = nullptr;
            t.xlo0 = bx.alloc.lo[0]; t.xlo1 = bx.alloc.lo[1]; t.xs = bx.st[0];
            t.mlo1 = 0; t.ylo0 = 0; t.ylo1 = 0; t.ys = 0;
            t.i0 = (int32_t)W.lo[0]; t.i1 = (int32_t)W.hi[0]; t.j0 = (int32_t)W.lo[1]; t.j1 = (int32_t)W.hi[1];
            t.n = (int32_t)X->n[0];
            t.mode = (k.kind == K_COLNORM || k.kind == K_COLSCALE) ? 1 : 0;
            if (k.kind != K_SYMM) {
                const DevBuf &bm = pl.args[1]->buf[p];
                t.m = bm.ptr;
                t.mlo1 = bm.alloc.lo[1];
            }
            if (!reduce_cols) {
                const DevBuf &by = pointwise ? pl.args[2]->buf[p] : bx;
                t.y = by.ptr;
                t.ylo0 = by.alloc.lo[0]; t.ylo1 = by.alloc.lo[1]; t.ys = by.st[0];
            }
            cov.push_back(t);
            max_rows = std::max<int>(max_rows, t.i1 - t.i0);
            max_cols = std::max<int>(max_cols, t.j1 - t.j0);
        } else if (k.kind == K_GEMM || k.kind == K_TRMM || k.kind == K_SYRK) {
            const bool syrk = k.kind == K_SYRK;  // A = X read transposed, B = X, C = the second argument
            HDArray *A = pl.args[0], *B = pl.args[0], *C = syrk ? pl.args[1] : pl.args[2];
            if (!syrk) B = pl.args[1];
            const DevBuf &ba = A->buf[p], &bb = B->buf[p], &bc = C->buf[p];
            GemmPart q;
            q.a = ba.ptr; q.b = bb.ptr; q.c = bc.ptr;
            q.alo0 = ba.alloc.lo[0]; q.alo1 = ba.alloc.lo[1]; q.as = ba.st[0];
            q.blo0 = bb.alloc.lo[0]; q.blo1 = bb.alloc.lo[1]; q.bs = bb.st[0];
            q.clo0 = bc.alloc.lo[0]; q.clo1 = bc.alloc.lo[1]; q.cs = bc.st[0];
            q.i0 = (int32_t)W.lo[0]; q.i1 = (int32_t)W.hi[0];
            q.j0 = (int32_t)W.lo[1]; q.j1 = (int32_t)W.hi[1];
            q.nk = (int32_t)(syrk ? A->n[0] : A->n[1]);
            q.lower = k.kind == K_TRMM ? 1 : 0;
            q.transa = syrk ? 1 : 0;
            q.upper = syrk ? 1 : 0;
            if (A->dtype == DT_F32) {  // tensor cores, bf16x3
                TcPart t;
                t.a = q.a; t.b = q.b; t.c = q.c;
                t.alo0 = q.alo0; t.alo1 = q.alo1; t.as = q.as;
                t.blo0 = q.blo0; t.blo1 = q.blo1; t.bs = q.bs;
                t.clo0 = q.clo0; t.clo1 = q.clo1; t.cs = q.cs;
                t.i1 = q.i1; t.j1 = q.j1; t.lower = q.lower; t.pad = 0;
                const int pi = (int)tp.size();
                tp.push_back(t);
                const int tcbn = 256;  // CTA tile width of both forms
                for (int ti = q.i0; ti < q.i1; ti += 128)
                    for (int tj = q.j0; tj < q.j1; tj += tcbn) {
                        if (q.upper && tj + tcbn - 1 < ti) continue;  // entirely below the diagonal
                        TcTile x;
                        x.part = pi; x.i0 = ti; x.j0 = tj;
                        x.kend = q.lower ? std::min(q.nk, std::min(ti + 128, q.i1)) : q.nk;
                        tt.push_back(x);
                    }
            } else {
                gp.push_back(q);
                max_rows = std::max<int>(max_rows, q.i1 - q.i0);
                max_cols = std::max<int>(max_cols, q.j1 - q.j0);
            }
        } else if (k.kind == K_EXCHANGE) {
            continue;
        } else {
            return HDARRAY_ERR_UNSUPPORTED;
        }
    }
    blobs.push_back({xfer.data(), xfer.size() * sizeof(CopyTask)});
    blobs.push_back({local.data(), local.size() * sizeof(CopyTask)});
    blobs.push_back({pw.data(), pw.size() * sizeof(PwTask)});
    blobs.push_back({gp.data(), gp.size() * sizeof(GemmPart)});
    // heaviest tiles first: CTAs start in index order, so the long ones do not end up last
    std::stable_sort(tt.begin(), tt.end(), [](const TcTile &x, const TcTile &y) { return x.kend > y.kend; });
    blobs.push_back({tp.data(), tp.size() * sizeof(TcPart)});
    blobs.push_back({tt.data(), tt.size() * sizeof(TcTile)});
    blobs.push_back({cov.data(), cov.size() * sizeof(CovTask)});
    std::vector<const char *> addr;
    int rc = upload(blobs, pl.tables, addr);
    if (rc) return rc;

    auto push_copy = [&](const CopyTask *base, const std::vector<std::pair<int, int>> &groups, int64_t total) {
        if (plain) {
            for (auto &gr : groups)
                if (gr.second > gr.first) {
                    LaunchRec L; L.kind = L_COPY; L.p0 = base + gr.first; L.n0 = gr.second - gr.first;
                    pl.launches.push_back(L);
                }
        } else if (total > 0) {
            LaunchRec L; L.kind = L_COPY; L.p0 = base; L.n0 = total;
            pl.launches.push_back(L);
        }
    };
    push_copy((const CopyTask *)addr[0], xfer_groups, (int64_t)xfer.size());
    push_copy((const CopyTask *)addr[1], local_groups, (int64_t)local.size());
    if (k.kind == K_USER && !pl.user_work.empty()) {
        LaunchRec L; L.kind = L_USER;
        L.p0 = pl.user_work.data(); L.n0 = (int64_t)pl.user_work.size();
        L.p1 = pl.scal.data(); L.n1 = (int64_t)pl.scal.size(); L.p2 = &k;
        pl.launches.push_back(L);
    }
    if (!cov.empty()) {
        LaunchRec L;
        L.kind = (k.kind == K_COLMEAN || k.kind == K_COLNORM) ? L_COLMEAN
                 : (k.kind == K_CENTER || k.kind == K_COLSCALE) ? L_CENTER : L_SYMM;
        L.dtype = pl.args[0]->dtype; L.p0 = addr[6]; L.n0 = (int64_t)cov.size(); L.n1 = max_rows; L.n2 = max_cols;
        pl.launches.push_back(L);
    }
    if (!pw.empty()) {
        auto add = [&](int b, int e, const void *red, int64_t nblocks) {
            LaunchRec L; L.kind = L_SQDIFF; L.dtype = pl.args[0]->dtype;
            L.p0 = (const PwTask *)addr[2] + b; L.n0 = e - b;
            L.p1 = red; L.n1 = nblocks;
            pl.launches.push_back(L);
        };
        if (plain) {
            for (auto &gr : pw_groups) add(gr.first, gr.second, nullptr, 0);
        } else {  // one launch that also folds the sum of R (read back by HDArrayReduce)
            const int64_t nb = std::min<int64_t>((int64_t)pw.size(), 4 * (int64_t)g->nsm);
            if (!pl.red || pl.red->bytes < red_bytes(nb)) {
                pl.red = std::make_shared<DevMem>();
                const int arc = dev_alloc(&pl.red->ptr, red_bytes(nb));
                if (arc) {
                    pl.red->ptr = nullptr;
                    return arc;
                }
                pl.red->bytes = red_bytes(nb);
                CUDA_TRY(cudaMemset(pl.red->ptr, 0, red_bytes(nb)));
            }
            add(0, (int)pw.size(), pl.red->ptr, nb);
        }
    }
    if (!gp.empty()) {
        auto add = [&](int b, int e, int mr, int mc) {
            LaunchRec L; L.kind = L_GEMM64;
            L.p0 = (const GemmPart *)addr[3] + b; L.n0 = e - b; L.n1 = mr; L.n2 = mc;
            L.f0 = pl.scal.size() > 0 ? pl.scal[0] : 1.0;
            L.f1 = pl.scal.size() > 1 ? pl.scal[1] : 0.0;
            pl.launches.push_back(L);
        };
        if (plain)
            for (size_t i = 0; i < gp.size(); i++) add((int)i, (int)i + 1, gp[i].i1 - gp[i].i0, gp[i].j1 - gp[i].j0);
        else
            add(0, (int)gp.size(), max_rows, max_cols);
    }
    // Panel path: split the operands once into pre-tiled bf16 panels (128-byte swizzled, K-major)
    // and stream them with bulk copies.  Each device's row range of A and column range of B get a
    // panel, split from that device's own buffer (after this call's exchange it holds those rows
    // of A and columns of B in full); devices with the same range share one panel (row blocks
    // share B, column blocks share A).
    bool panel_ok = !tt.empty();
    for (const TcPart &t : tp) panel_ok = panel_ok && t.j1 > 0;
    const bool syrk = k.kind == K_SYRK;  // only the panel kernel reads A transposed
    const int nsp = g->gemm_parts;       // bf16 parts per value (3: only the panel kernel has it)
    const int tcbn = 256;                // CTA tile width
    const int pbk = nsp == 3 ? 32 : 64;  // K per panel tile (64-byte or 128-byte rows)
    if (panel_ok && (syrk || nsp == 3 || getenv("HDARRAY_GEMM_NO_PANELS") == nullptr)) {
        HDArray *A = pl.args[0], *B = syrk ? pl.args[0] : pl.args[1];
        const int64_t nk = syrk ? A->n[0] : A->n[1];
        const int nkt_b = (int)((nk + pbk - 1) / pbk);
        std::vector<SplitJob> ajobs, bjobs;
        std::vector<PanelPart> pp;
        std::map<std::pair<int64_t, int64_t>, size_t> aoff, boff;
        size_t total = 0;
        for (int p = 0; p < pt.nparts; p++) {
            const Box &W = pt.box[p];
            if (W.empty()) continue;
            const int64_t kend = (k.kind == K_TRMM) ? std::min<int64_t>(nk, W.hi[0]) : nk;
            const int nkt = (int)((kend + pbk - 1) / pbk);
            const auto ka = std::make_pair(W.lo[0], W.hi[0]), kb = std::make_pair(W.lo[1], W.hi[1]);
            if (!aoff.count(ka)) {
                const int nmt = (int)((W.hi[0] - W.lo[0] + 127) / 128);
                aoff[ka] = total;
                total += (size_t)nmt * nkt * nsp * (128 * pbk * 2);
                SplitJob J;
                const DevBuf &ba = A->buf[p];
                J.src = ba.ptr; J.dst = (void *)(uintptr_t)aoff[ka];  // offset until the panels exist
                J.lo0 = ba.alloc.lo[0]; J.lo1 = ba.alloc.lo[1]; J.stride = ba.st[0];
                J.row0 = (int32_t)W.lo[0]; J.row_end = (int32_t)W.hi[0]; J.kend = (int32_t)kend;
                J.nkt = nkt; J.ntiles = nmt * nkt; J.rows_per_tile = 128; J.transpose = syrk ? 1 : 0;
                J.lower = k.kind == K_TRMM ? 1 : 0;
                J.nparts = nsp;
                J.bk = pbk;
                ajobs.push_back(J);
            }
            if (!boff.count(kb)) {
                const int nnt = (int)((W.hi[1] - W.lo[1] + tcbn - 1) / tcbn);
                boff[kb] = total;
                total += (size_t)nnt * nkt_b * nsp * ((size_t)tcbn * pbk * 2);
                SplitJob J;
                const DevBuf &bb = B->buf[p];
                J.src = bb.ptr; J.dst = (void *)(uintptr_t)boff[kb];
                J.lo0 = bb.alloc.lo[0]; J.lo1 = bb.alloc.lo[1]; J.stride = bb.st[0];
                J.row0 = (int32_t)W.lo[1]; J.row_end = (int32_t)W.hi[1]; J.kend = (int32_t)nk;
                J.nkt = nkt_b; J.ntiles = nnt * nkt_b; J.rows_per_tile = tcbn; J.transpose = 1; J.lower = 0;
                J.nparts = nsp;
                J.bk = pbk;
                bjobs.push_back(J);
            }
            PanelPart q;
            const TcPart &t = tp[pp.size()];
            q.apanel = (const void *)(uintptr_t)aoff[ka];
            q.bpanel = (const void *)(uintptr_t)boff[kb];
            q.c = t.c;
            q.clo0 = t.clo0; q.clo1 = t.clo1; q.cs = t.cs;
            q.row0 = (int32_t)W.lo[0]; q.col0 = (int32_t)W.lo[1];
            q.i1 = (int32_t)W.hi[0]; q.j1 = (int32_t)W.hi[1];
            q.nkt = nkt; q.nkt_b = nkt_b;
            q.upper = syrk ? 1 : 0; q.nparts = nsp;
            pp.push_back(q);
        }
        auto panels = std::make_shared<DevMem>();
        {
            const int arc = dev_alloc(&panels->ptr, total);
            if (arc) {
                panels->ptr = nullptr;
                return arc;
            }
        }
        panels->bytes = total;
        char *base = (char *)panels->ptr;
        for (SplitJob &J : ajobs) J.dst = base + (uintptr_t)J.dst;
        for (SplitJob &J : bjobs) J.dst = base + (uintptr_t)J.dst;
        for (PanelPart &q : pp) {
            q.apanel = base + (uintptr_t)q.apanel;
            q.bpanel = base + (uintptr_t)q.bpanel;
        }
        // tiles index the PanelPart table in the same order as TcPart
        std::vector<std::pair<const void *, size_t>> pb = {
            {ajobs.data(), ajobs.size() * sizeof(SplitJob)}, {bjobs.data(), bjobs.size() * sizeof(SplitJob)},
            {pp.data(), pp.size() * sizeof(PanelPart)}, {tt.data(), tt.size() * sizeof(TcTile)}};
        std::shared_ptr<DevMem> ptab;
        std::vector<const char *> pa;
        int rc2 = upload(pb, ptab, pa);
        if (rc2) return rc2;
        int amax = 0, bmax = 0;
        for (const SplitJob &J : ajobs) amax = std::max(amax, J.ntiles);
        for (const SplitJob &J : bjobs) bmax = std::max(bmax, J.ntiles);
        LaunchRec SA; SA.kind = L_SPLIT; SA.p0 = pa[0]; SA.n0 = (int64_t)ajobs.size(); SA.n1 = amax; SA.n3 = 0;
        LaunchRec SB; SB.kind = L_SPLIT; SB.p0 = pa[1]; SB.n0 = (int64_t)bjobs.size(); SB.n1 = bmax; SB.n3 = 1;
        LaunchRec GM; GM.kind = L_GEMM_PANEL; GM.p0 = pa[2]; GM.p1 = pa[3]; GM.p2 = g->err_word;
        GM.n0 = (int64_t)tt.size();
        GM.n1 = nsp;
        GM.n3 = (int64_t)g->spin_limit;
        GM.f0 = pl.scal.size() > 0 ? pl.scal[0] : 1.0;
        GM.f1 = pl.scal.size() > 1 ? pl.scal[1] : 0.0;
        pl.launches.push_back(SA);
        pl.launches.push_back(SB);
        pl.launches.push_back(GM);
        pl.panels = panels;
        pl.split_version[0] = pl.split_version[1] = ~0ull;
        pl.extra_tables = ptab;
        tt.clear();
    }
    if (!tt.empty()) {
        LaunchRec L; L.kind = L_GEMM_TC;
        L.p0 = addr[4]; L.p1 = addr[5]; L.p2 = g->err_word; L.n0 = (int64_t)tt.size();
        L.f0 = pl.scal.size() > 0 ? pl.scal[0] : 1.0;
        L.f1 = pl.scal.size() > 1 ? pl.scal[1] : 0.0;
        pl.launches.push_back(L);
    }
    pl.copy_host = xfer;
    return HDARRAY_OK;
}

// ------------------------------------------------------------------------------------------
// Issuing launches (directly, into a batch, or into a graph recording)
// ------------------------------------------------------------------------------------------

int issue_recorded(const LaunchRec &L)
{
    cudaError_t e = issue(L, g->stream);
    if (e != cudaSuccess) {
        if (L.kind == L_USER) return user_launch_rc();  // the user launcher's own code
        if (trace()) fprintf(stderr, "hdarray: launch failed: %s\n", cudaGetErrorString(e));
        return HDARRAY_ERR_CUDA;
    }
    g->counters[0]++;
    if (g->recording) g->rec.push_back(L);
    return HDARRAY_OK;
}

int run_plan(const std::shared_ptr<Plan> &pl)
{
    if (g->host_only) return HDARRAY_OK;
    bool alternated = false;
    for (const LaunchRec &L : pl->launches) {
        if (L.kind == L_SPLIT) {  // panels of an operand whose content has not changed are reused
            const int which = (int)L.n3;
            const uint64_t v = pl->args[which]->version;
            if (!g->recording && pl->split_version[which] == v) continue;
            pl->split_version[which] = v;
        }
        int rc;
        if (L.p1_alt && L.alt_calls) {  // every other call of the plan takes its reversed tile table
            LaunchRec M = L;
            if (pl->alt) M.p1 = L.p1_alt;
            M.p1_alt = nullptr;
            rc = issue_recorded(M);
            alternated = true;
        } else {
            rc = issue_recorded(L);
        }
        if (rc) return rc;
    }
    if (alternated) pl->alt = !pl->alt;
    if (g->recording) g->rec_refs.push_back(pl);
    return HDARRAY_OK;
}

int flush_batch();

// ------------------------------------------------------------------------------------------
// Autotuner: tile shapes of the fused stencil launches
// ------------------------------------------------------------------------------------------

std::string tune_key(const Plan &pl)
{
    const Part &pt = g->parts[pl.part];
    std::string k = pl.k->name + ":" + std::to_string(pl.args[0]->dtype) + ":" + std::to_string(pt.nparts);
    for (const Box &b : pt.box) {
        char buf[96];
        snprintf(buf, sizeof(buf), ":%lld,%lld,%lld", (long long)(b.hi[0] - b.lo[0]), (long long)(b.hi[1] - b.lo[1]),
                 (long long)(b.hi[2] - b.lo[2]));
        k += buf;
    }
    return k;
}

void apply_shape(const Ctx::Shape &s, bool threed)
{
    g->fuse = s.fuse;
    if (threed) {
        g->tile_z = s.tile_z;
        g->variant3 = s.variant3;
        g->tile_rows = s.rows;
        g->band3 = s.band3;
        g->cta3 = s.cta3;
    } else {
        g->variant = s.variant;
        g->tile_rows = s.rows;
        g->warps_per_cta = s.warps;
        g->band2 = s.band2;
    }
}

Ctx::Shape current_shape()
{
    return Ctx::Shape{g->variant, g->tile_rows, g->warps_per_cta, g->tile_z, g->fuse, g->variant3, g->band3, g->cta3, g->band2};
}

const char *tune_file() { return getenv("HDARRAY_TUNE_CACHE"); }

void load_tune_file()
{
    if (g->tune_file_loaded || !tune_file()) return;
    g->tune_file_loaded = true;
    FILE *f = fopen(tune_file(), "r");
    if (!f) return;
    char key[4096];
    Ctx::Shape s;
    while (fscanf(f, "%4095s %d %d %d %d %d %d %d %d %d", key, &s.variant, &s.rows, &s.warps, &s.tile_z, &s.fuse,
                  &s.variant3, &s.band3, &s.cta3, &s.band2) == 10)
        g->tuned[key] = s;
    fclose(f);
}

void save_tune(const std::string &key, const Ctx::Shape &s)
{
    if (!tune_file()) return;
    FILE *f = fopen(tune_file(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d %d\n", key.c_str(), s.variant, s.rows, s.warps, s.tile_z, s.fuse,
            s.variant3, s.band3, s.cta3, s.band2);
    fclose(f);
}

float time_plan(const Plan &pl, int reps)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        cudaGetLastError();
        return 1e30f;
    }
    float best = 1e30f;
    for (int r = 0; r < reps + 1; r++) {
        cudaEventRecord(a, g->stream);
        for (const LaunchRec &L0 : pl.launches) {
            LaunchRec L = L0;  // successive runs alternate the tile order, as iterations do
            if (L.p1_alt && (r & 1)) L.p1 = L.p1_alt;
            if (issue(L, g->stream) != cudaSuccess) {
                cudaGetLastError();
                best = 1e30f;
                r = reps + 1;
                break;
            }
        }
        cudaEventRecord(b, g->stream);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0 && ms < best) best = ms;  // the first run warms up
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

int compile_plan(Plan &pl);

// Compile a fused stencil plan with the best tile shape for its partition, timing the candidates
// on the GPU the first time a shape key is seen.  Re-running the launch is harmless: it recomputes
// Y from an unchanged X and copies the same halo values again.
int compile_tuned(Plan &pl)
{
    const bool stencil = pl.k->kind == K_JACOBI2D || pl.k->kind == K_STENCIL3D || pl.k->kind == K_CONV2D;
    if (!stencil || !g->autotune || g->recording || g->batching || g->tuning) return compile_plan(pl);
    const bool threed = pl.k->kind == K_STENCIL3D;
    load_tune_file();
    const std::string key = tune_key(pl);
    const Ctx::Shape saved = current_shape();
    auto it = g->tuned.find(key);
    if (it != g->tuned.end()) {
        apply_shape(it->second, threed);
        int rc = compile_plan(pl);
        apply_shape(saved, threed);
        return rc;
    }
    g->fuse = 1;  // probe: does this plan's exchange fit the tiles (its steady form)?
    int rc = compile_plan(pl);
    g->fuse = saved.fuse;
    if (rc || !pl.fused) return rc ? rc : compile_plan(pl);  // tune on the steady form only
    std::vector<Ctx::Shape> cands;
    const bool flat_ok = pl.args[0]->dtype != DT_BF16;
    if (threed) {
        for (int fu : {1, 0})
            for (int tz : {16, 32, 64}) {
                for (int v3 : {1, 3})
                    for (int band : {16, 32, 64})
                        for (int cta : {256, 512})
                            cands.push_back(Ctx::Shape{saved.variant, saved.rows, saved.warps, tz, fu, v3, band, cta,
                                                       saved.band2});
                if (flat_ok)
                    for (int cells : {16, 32})
                        cands.push_back(Ctx::Shape{saved.variant, cells, saved.warps, tz, fu, 2, saved.band3, saved.cta3,
                                                   saved.band2});
            }
    } else if (pl.k->kind == K_CONV2D) {  // the packed-stream kernel, or rows staged by TMA
        for (int fu : {1, 0}) {
            for (int band : {8, 16, 32})
                for (int rows : {16, 32, 64})
                    cands.push_back(Ctx::Shape{3, rows, saved.warps, saved.tile_z, fu, saved.variant3,
                                               saved.band3, saved.cta3, band});
            for (int band : {16, 32, 64})
                for (int rows : {8, 16, 24})
                    cands.push_back(Ctx::Shape{5, rows, saved.warps, saved.tile_z, fu, saved.variant3,
                                               saved.band3, saved.cta3, band});
        }
    } else {
        int64_t cells = 0;  // short tiles (more warps) are candidates for small grids only
        for (int p = 0; p < g->parts[pl.part].nparts; p++) cells += g->parts[pl.part].box[p].volume();
        const std::vector<int> row_cands = cells < (1 << 22) ? std::vector<int>{4, 8, 16, 32, 64}
                                                              : std::vector<int>{16, 32, 64};
        for (int fu : {1, 0}) {
            for (int v : {0, 1})
                for (int rows : row_cands)
                    for (int w : {4, 8})
                        cands.push_back(Ctx::Shape{v, rows, w, saved.tile_z, fu, saved.variant3, saved.band3, saved.cta3,
                                                   saved.band2});
            for (int band : {8, 16, 32})
                for (int rows : {16, 32, 64})
                    cands.push_back(Ctx::Shape{3, rows, saved.warps, saved.tile_z, fu, saved.variant3, saved.band3, saved.cta3,
                                               band});
            // rows staged by TMA: tiles of about 8 * rows rows (longer tiles measured slower in every
            // steady-state run, though a single timing sometimes ranked them first)
            for (int band : {16, 32, 64})
                for (int rows : {8, 16})
                    cands.push_back(Ctx::Shape{5, rows, saved.warps, saved.tile_z, fu, saved.variant3, saved.band3, saved.cta3,
                                               band});
            if (flat_ok)
                for (int cells : {16, 32, 64})
                    cands.push_back(Ctx::Shape{2, cells, saved.warps, saved.tile_z, fu, saved.variant3, saved.band3, saved.cta3,
                                               saved.band2});
        }
    }
    g->tuning = true;
    std::vector<std::pair<float, Ctx::Shape>> timed;
    float best_ms = 1e30f;
    for (const Ctx::Shape &c : cands) {
        apply_shape(c, threed);
        if (compile_plan(pl) != HDARRAY_OK) continue;
        const float ms = time_plan(pl, 7);
        timed.push_back({ms, c});
        best_ms = std::min(best_ms, ms);
    }
    // the shapes within 5% of the fastest are timed again over three times as many launches, and
    // only they stay in the running: one short timing of each shape alone picked different shapes
    // from run to run where several were close
    {
        std::vector<std::pair<float, Ctx::Shape>> finalists;
        float again = 1e30f;
        for (const auto &tc : timed) {
            if (tc.first > best_ms * 1.05f) continue;
            apply_shape(tc.second, threed);
            if (compile_plan(pl) != HDARRAY_OK) continue;
            const float ms = time_plan(pl, 21);
            finalists.push_back({ms, tc.second});
            again = std::min(again, ms);
        }
        if (!finalists.empty()) {
            timed.swap(finalists);
            best_ms = again;
        }
    }
    // single launches time a plan alone; in an iteration the 2-D launches alternate their tile
    // order and the shorter tiles make the better use of that, so among 2-D shapes within 2% of
    // the fastest take the one with the shortest tiles (then the fastest)
    Ctx::Shape best = saved;
    float pick_ms = 1e30f;
    int pick_rows = 1 << 30;
    const float slack = threed ? 1.0f : 1.02f;
    for (const auto &tc : timed) {
        if (tc.first > best_ms * slack) continue;
        const int r = threed ? 0 : tc.second.rows;
        if (r < pick_rows || (r == pick_rows && tc.first < pick_ms)) {
            pick_rows = r;
            pick_ms = tc.first;
            best = tc.second;
        }
    }
    g->tuning = false;
    apply_shape(best, threed);
    rc = compile_plan(pl);
    apply_shape(saved, threed);
    g->tuned[key] = best;
    save_tune(key, best);
    if (trace())
        fprintf(stderr, "hdarray: tuned %s -> variant %d/%d rows %d warps %d tile_z %d band %d/%d cta %d fuse %d (%.1f us)\n",
                key.c_str(), best.variant, best.variant3, best.rows, best.warps, best.tile_z, best.band2, best.band3,
                best.cta3, best.fuse, pick_ms * 1e3);
    return rc;
}

// ------------------------------------------------------------------------------------------
// Applying a kernel
// ------------------------------------------------------------------------------------------

int validate_args(const KernelDef &k, const Part &pt, const std::vector<HDArray *> &a)
{
    for (HDArray *x : a)
        if (!x || !g->arrays.count(x)) return HDARRAY_ERR_INVAL;
    const HDArray *sp = a[k.space];
    if (pt.dim != sp->dim) return HDARRAY_ERR_INVAL;
    for (int d = 0; d < 3; d++)
        if (pt.n[d] != sp->n[d]) return HDARRAY_ERR_INVAL;
    auto same = [](const HDArray *x, const HDArray *y) {
        return x->dim == y->dim && x->n[0] == y->n[0] && x->n[1] == y->n[1] && x->n[2] == y->n[2];
    };
    switch (k.kind) {
    case K_JACOBI2D:
    case K_CONV2D:
    case K_STENCIL3D:
        if (a[0] == a[1] || !same(a[0], a[1]) || a[0]->dtype != a[1]->dtype) return HDARRAY_ERR_INVAL;
        if (a[0]->dim != (k.kind == K_STENCIL3D ? 3 : 2)) return HDARRAY_ERR_INVAL;
        for (int p = 0; p < pt.nparts; p++) {  // every work element needs all its neighbours
            const Box &w = pt.box[p];
            if (w.empty()) continue;
            for (int d = 0; d < a[0]->dim; d++)
                if (w.lo[d] < 1 || w.hi[d] > a[0]->n[d] - 1) return HDARRAY_ERR_RANGE;
        }
        break;
    case K_COPY:
        if (a[0] == a[1] || !same(a[0], a[1]) || a[0]->dtype != a[1]->dtype) return HDARRAY_ERR_INVAL;
        break;
    case K_SQDIFF:
        if (!same(a[0], a[1]) || !same(a[0], a[2]) || a[0]->dtype != a[1]->dtype) return HDARRAY_ERR_INVAL;
        if (a[2]->dtype != DT_F64 || a[2] == a[0] || a[2] == a[1]) return HDARRAY_ERR_INVAL;
        break;
    case K_EXCHANGE:
        break;
    case K_COLMEAN:
    case K_COLNORM:
    case K_COLSCALE:
    case K_CENTER: {
        const HDArray *X = a[0], *M = a[1];
        if (X->dim != 2 || M->dim != 2 || M->n[0] != 1 || M->n[1] != X->n[1] || X == M) return HDARRAY_ERR_INVAL;
        if (X->dtype != M->dtype || (X->dtype != DT_F64 && X->dtype != DT_F32)) return HDARRAY_ERR_INVAL;
        if (k.kind == K_CENTER || k.kind == K_COLSCALE) {
            const HDArray *Y = a[2];
            if (!same(X, Y) || Y == X || Y == M || Y->dtype != X->dtype) return HDARRAY_ERR_INVAL;
        }
        break;
    }
    case K_SYRK: {
        const HDArray *X = a[0], *C = a[1];
        if (X->dim != 2 || C->dim != 2 || C->n[0] != X->n[1] || C->n[1] != X->n[1] || C == X) return HDARRAY_ERR_INVAL;
        if (X->dtype != C->dtype || (X->dtype != DT_F64 && X->dtype != DT_F32)) return HDARRAY_ERR_INVAL;
        break;
    }
    case K_SYMM:
        if (a[0]->dim != 2 || a[0]->n[0] != a[0]->n[1]) return HDARRAY_ERR_INVAL;
        break;
    case K_USER:
        if (k.narr > HDARRAY_MAX_KERNEL_ARRAYS || !k.launcher) return HDARRAY_ERR_INVAL;
        break;
    case K_GEMM:
    case K_TRMM: {
        const HDArray *A = a[0], *B = a[1], *C = a[2];
        if (A->dim != 2 || B->dim != 2 || C->dim != 2) return HDARRAY_ERR_INVAL;
        if (A->n[0] != C->n[0] || A->n[1] != B->n[0] || B->n[1] != C->n[1]) return HDARRAY_ERR_INVAL;
        if (C == A || C == B) return HDARRAY_ERR_INVAL;
        if (A->dtype != B->dtype || A->dtype != C->dtype) return HDARRAY_ERR_INVAL;
        if (A->dtype == DT_BF16) return HDARRAY_ERR_UNSUPPORTED;  // binary64 (DFMA) or binary32 (bf16x3)
        break;
    }
    }
    return HDARRAY_OK;
}

int apply(const char *kname, int part, const std::vector<HDArray *> &args, const std::vector<double> &scal)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!kname) return HDARRAY_ERR_INVAL;
    auto kit = g->kernels.find(kname);
    if (kit == g->kernels.end()) return HDARRAY_ERR_INVAL;
    const KernelDef &k = kit->second;
    if (part < 0 || part >= (int)g->parts.size()) return HDARRAY_ERR_INVAL;
    if ((int)args.size() != k.narr) return HDARRAY_ERR_INVAL;
    const Part &pt = g->parts[part];
    int rc = validate_args(k, pt, args);
    if (rc) return rc;
    for (HDArray *a : args) grow_devices(a, pt.nparts);
    if (!g->host_only)
        for (HDArray *a : args) {
            rc = join_write(a);
            if (rc) return rc;
        }

    std::vector<uint64_t> absv(args.size(), 0);
    std::vector<const Ctx::AbsSpec *> abss(args.size(), nullptr);
    for (size_t i = 0; i < args.size(); i++) {
        auto it = g->abs.find(std::make_tuple(k.name, part, args[i]->uid));
        if (it != g->abs.end()) {
            absv[i] = it->second.version;
            abss[i] = &it->second;
        }
    }
    const std::string key = memo_key(k, part, args, absv, scal);
    std::shared_ptr<Plan> pl;
    auto mit = g->memo.find(key);
    if (mit != g->memo.end()) {
        pl = mit->second;
        g->counters[3]++;
    } else {
        pl = std::make_shared<Plan>();
        pl->id = g->next_plan++;
        pl->k = &k;
        pl->part = part;
        pl->args = args;
        pl->scal = scal;
        pl->luse.resize(args.size());
        pl->ldef.resize(args.size());
        for (size_t i = 0; i < args.size(); i++) {
            const auto *au = abss[i] && abss[i]->has_use ? &abss[i]->use : nullptr;
            const auto *ad = abss[i] && abss[i]->has_def ? &abss[i]->def : nullptr;
            clause_sets(pt, args[i], k.use[i], au, pl->luse[i]);
            clause_sets(pt, args[i], k.def[i], ad, pl->ldef[i]);
        }
        // one step per distinct array: union of its arguments' sections
        for (size_t i = 0; i < args.size(); i++) {
            bool seen = false;
            for (ArrStep &st : pl->steps) seen = seen || st.a == args[i];
            if (seen) continue;
            ArrStep st;
            st.a = args[i];
            std::vector<BoxSet> U(pt.nparts), D(pt.nparts);
            for (size_t j = i; j < args.size(); j++) {
                if (args[j] != args[i]) continue;
                for (int p = 0; p < pt.nparts; p++) {
                    U[p] = set_union(U[p], pl->luse[j][p]);
                    D[p] = set_union(D[p], pl->ldef[j][p]);
                }
            }
            for (int p = 0; p < pt.nparts; p++) {
                st.used = st.used || !U[p].empty();
                st.defined = st.defined || !D[p].empty();
            }
            GState s = args[i]->states[args[i]->cur];
            st.pre = args[i]->cur;
            rc = use_step(s, U, st.moves);
            if (rc) return rc;
            rc = def_step(s, D);
            if (rc) return rc;
            st.post = intern(args[i], std::move(s));
            pl->steps.push_back(std::move(st));
        }
        if (g->memo.size() >= 16384) g->memo.clear();  // bounded; plans held by graphs stay alive
        g->memo[key] = pl;
        g->counters[2]++;
        if (trace()) {
            int64_t nb = 0;
            for (auto &st : pl->steps) for (auto &m : st.moves) nb += m.box.volume() * st.a->esize;
            fprintf(stderr, "hdarray: plan %llu for %s part %d: %lld bytes to move\n",
                    (unsigned long long)pl->id, k.name.c_str(), part, (long long)nb);
        }
    }
    // calls of one batch must be independent: refuse one that touches what another defines
    if (g->batching) {
        for (const ArrStep &st : pl->steps) {
            if (g->batch_defined.count(st.a)) return HDARRAY_ERR_RACE;
            if (st.defined && g->batch_used.count(st.a)) return HDARRAY_ERR_RACE;
        }
        for (const ArrStep &st : pl->steps) {
            if (st.defined) g->batch_defined.insert(st.a);
            else g->batch_used.insert(st.a);
        }
    }
    // buffers must cover every device's sections before anything is compiled or launched
    if (!g->host_only) {
        for (size_t i = 0; i < args.size(); i++) {
            for (int p = 0; p < pt.nparts; p++) {
                if (!is_local(p)) continue;  // another rank's device: no buffer here
                Box need = box_hull(set_bbox(pl->luse[i][p]), set_bbox(pl->ldef[i][p]));
                if (need.empty()) continue;
                if (g->batching && !(args[i]->buf[p].ptr && box_contains(args[i]->buf[p].alloc, need))) {
                    rc = flush_batch();
                    if (rc) return rc;
                }
                rc = ensure_buffer(args[i], p, need);
                if (rc) return rc;
            }
        }
        // a plan may be shared by signatures whose buffers moved: recompile when they did
        const std::string sig = epoch_sig(*pl);
        if (pl->compiled_sig != sig) {
            rc = compile_tuned(*pl);
            if (rc) return rc;
            pl->compiled_sig = sig;
        }
    }
    // bookkeeping moves on; the GPU work is issued now or at the end of the batch
    for (ArrStep &st : pl->steps) {
        if (g->recording && !g->rec_pre.count(st.a)) g->rec_pre[st.a] = {st.a->cur, st.a->generation};
        if (g->recording && st.defined) g->rec_defined.insert(st.a);
        st.a->cur = st.post;
        if (st.defined) st.a->version++;
        if (st.used) st.a->last_moves = st.moves;
        for (const Move &m : st.moves) g->counters[1] += m.box.volume() * st.a->esize;
    }
    for (const ArrStep &st : pl->steps) {  // sections that cross ranks arrive before the kernel
        rc = run_transport(st.a, st.moves);
        if (rc) return rc;
    }
    if (g->batching) {
        g->batch.push_back(pl);
        return HDARRAY_OK;
    }
    rc = run_plan(pl);
    if (rc) return rc;
    for (const ArrStep &st : pl->steps) {
        rc = note_use(st.a);
        if (rc) return rc;
    }
    if (k.kind == K_SQDIFF && pl->red && !g->host_only) {
        // the launch left the sum of R's new values over the work boxes in the plan's scratch
        for (const LaunchRec &L : pl->launches) {
            if (L.kind != L_SQDIFF || !L.p1) continue;
            g->sq_sum.R = args[2];
            g->sq_sum.version = args[2]->version;
            g->sq_sum.boxes = pt.box;
            g->sq_sum.pl = pl;
            g->sq_sum.sum = (const double *)((const char *)L.p1 + red_counter_offset(L.n1) + 128);
        }
    }
    return HDARRAY_OK;
}

// ------------------------------------------------------------------------------------------
// Batches: independent calls fused into as few launches as possible
// ------------------------------------------------------------------------------------------

int flush_batch()
{
    std::vector<std::shared_ptr<Plan>> plans;
    plans.swap(g->batch);
    if (plans.empty() || g->host_only) return HDARRAY_OK;
    // hazards: a defined array may appear in no other call of the batch
    for (size_t i = 0; i < plans.size(); i++)
        for (const ArrStep &si : plans[i]->steps) {
            if (!si.defined) continue;
            for (size_t j = 0; j < plans.size(); j++) {
                if (j == i) continue;
                for (const ArrStep &sj : plans[j]->steps)
                    if (sj.a == si.a) return HDARRAY_ERR_RACE;
            }
        }
    std::string key;
    char buf[64];
    for (auto &p : plans) {
        snprintf(buf, sizeof(buf), "%llu/%s;", (unsigned long long)p->id, p->compiled_sig.c_str());
        key += buf;
    }
    auto it = g->batch_cache.find(key);
    if (it == g->batch_cache.end()) {
        // merge: all exchanges first, then every fused 2-D stencil of the same type, then the rest
        std::vector<CopyTask> copies;
        std::map<std::tuple<int, int, int>, Sten2DHost> sten;  // (dtype, variant, warps)
        std::vector<LaunchRec> rest;
        // the calls X -> Y and Y -> X of a batch run their instances in opposite orders (each
        // plan's own tiles are reversed already), so an iteration starts where the last one ended
        std::vector<std::shared_ptr<Plan>> order(plans);
        if (g->snake && !order.empty() && order[0]->args.size() >= 2 && order[0]->args[0]->uid > order[0]->args[1]->uid)
            std::reverse(order.begin(), order.end());
        for (auto &p : order) {
            if (p->k->kind == K_JACOBI2D && g->mode == HDARRAY_MODE_FUSED) {
                copies.insert(copies.end(), p->copy_host.begin(), p->copy_host.end());
                Sten2DHost &h = sten[std::make_tuple(p->s2.dtype, p->s2.variant, p->s2.warps)];
                h.dtype = p->s2.dtype;
                h.flat = p->s2.flat;
                h.variant = p->s2.variant;
                h.warps = p->s2.warps;
                h.smem = std::max(h.smem, p->s2.smem);
                h.rx_cap = std::max(h.rx_cap, p->s2.rx_cap);
                const int pbase = (int)h.parts.size(), sbase = (int)h.segs.size();
                h.parts.insert(h.parts.end(), p->s2.parts.begin(), p->s2.parts.end());
                h.maps.insert(h.maps.end(), p->s2.maps.begin(), p->s2.maps.end());  // TMA: one per part
                h.segs.insert(h.segs.end(), p->s2.segs.begin(), p->s2.segs.end());
                for (StenTile2D t : p->s2.tiles) {
                    t.part += pbase;
                    t.seg0 += sbase;
                    h.tiles.push_back(t);
                }
            } else {
                rest.insert(rest.end(), p->launches.begin(), p->launches.end());
            }
        }
        std::vector<std::pair<const void *, size_t>> blobs;
        blobs.push_back({copies.data(), copies.size() * sizeof(CopyTask)});
        for (auto &kv : sten) {
            blobs.push_back({kv.second.parts.data(), kv.second.parts.size() * sizeof(StenPart2D)});
            blobs.push_back({kv.second.tiles.data(), kv.second.tiles.size() * sizeof(StenTile2D)});
            blobs.push_back({kv.second.segs.data(), kv.second.segs.size() * sizeof(Seg)});
            blobs.push_back({kv.second.maps.data(), kv.second.maps.size() * sizeof(CUtensorMap)});
        }
        std::shared_ptr<DevMem> mem;
        std::vector<const char *> addr;
        int rc = upload(blobs, mem, addr);
        if (rc) return rc;
        std::vector<LaunchRec> ls;
        if (!copies.empty()) {
            LaunchRec L; L.kind = L_COPY; L.p0 = addr[0]; L.n0 = (int64_t)copies.size();
            ls.push_back(L);
        }
        int ai = 1;
        for (auto &kv : sten) {
            LaunchRec L; L.kind = kv.second.flat ? L_FLAT2D : L_JACOBI2D; L.dtype = kv.second.dtype;
            L.p0 = addr[ai]; L.p1 = addr[ai + 1]; L.p2 = addr[ai + 2]; L.p3 = addr[ai + 3];
            L.n0 = (int64_t)kv.second.tiles.size();
            L.n1 = kv.second.flat ? (int64_t)kv.second.smem : kv.second.variant == 5 ? kv.second.rx_cap : kv.second.warps;
            L.n2 = kv.second.variant;
            L.n3 = (int64_t)kv.second.smem;
            ai += 4;
            if (L.n0 > 0) ls.push_back(L);
        }
        ls.insert(ls.end(), rest.begin(), rest.end());
        if (g->batch_cache.size() > 64) g->batch_cache.clear();
        it = g->batch_cache.emplace(key, std::make_pair(mem, ls)).first;
    }
    for (const LaunchRec &L : it->second.second) {
        int rc = issue_recorded(L);
        if (rc) return rc;
    }
    if (g->recording) {
        g->rec_mems.push_back(it->second.first);
        for (auto &p : plans) g->rec_refs.push_back(p);
    }
    for (auto &p : plans)
        for (const ArrStep &st : p->steps) {
            int rc = note_use(st.a);
            if (rc) return rc;
        }
    return HDARRAY_OK;
}

// ------------------------------------------------------------------------------------------
// Data movement between user arrays and device buffers (Write / Read / Reduce)
// ------------------------------------------------------------------------------------------

int check_part_for(const HDArray *a, int part)
{
    if (part < 0 || part >= (int)g->parts.size()) return HDARRAY_ERR_INVAL;
    const Part &pt = g->parts[part];
    if (pt.dim != a->dim) return HDARRAY_ERR_INVAL;
    for (int d = 0; d < 3; d++)
        if (pt.n[d] != a->n[d]) return HDARRAY_ERR_INVAL;
    return HDARRAY_OK;
}

int check_device_error();

// host/device user array (dense, full size) <-> device buffer, one box
int memcpy_box(const HDArray *a, const DevBuf &b, const Box &bx, void *user, bool to_device)
{
    const int64_t es = a->esize;
    int64_t un[3], upos[3], bn[3], bpos[3], ext[3];
    // map to (width = innermost, height = middle, depth = outer) for cudaMemcpy3D
    int in = a->dim - 1;
    int mid = a->dim >= 2 ? a->dim - 2 : -1;
    int out = a->dim >= 3 ? 0 : -1;
    auto pick = [&](int d, const int64_t *v, int64_t dflt) { return d >= 0 ? v[d] : dflt; };
    ext[0] = (bx.hi[in] - bx.lo[in]) * es;
    ext[1] = mid >= 0 ? bx.hi[mid] - bx.lo[mid] : 1;
    ext[2] = out >= 0 ? bx.hi[out] - bx.lo[out] : 1;
    un[0] = a->n[in] * es;
    un[1] = pick(mid, a->n, 1);
    upos[0] = bx.lo[in] * es;
    upos[1] = mid >= 0 ? bx.lo[mid] : 0;
    upos[2] = out >= 0 ? bx.lo[out] : 0;
    const int64_t bw = (b.alloc.hi[in] - b.alloc.lo[in]);
    bn[0] = bw * es;
    bn[1] = mid >= 0 ? b.alloc.hi[mid] - b.alloc.lo[mid] : 1;
    bpos[0] = (bx.lo[in] - b.alloc.lo[in]) * es;
    bpos[1] = mid >= 0 ? bx.lo[mid] - b.alloc.lo[mid] : 0;
    bpos[2] = out >= 0 ? bx.lo[out] - b.alloc.lo[out] : 0;
    cudaMemcpy3DParms prm;
    memset(&prm, 0, sizeof(prm));
    cudaPitchedPtr up = make_cudaPitchedPtr(user, (size_t)un[0], (size_t)(un[0] / es), (size_t)un[1]);
    cudaPitchedPtr bp = make_cudaPitchedPtr(b.ptr, (size_t)bn[0], (size_t)bw, (size_t)bn[1]);
    cudaPos uo = make_cudaPos((size_t)upos[0], (size_t)upos[1], (size_t)upos[2]);
    cudaPos bo = make_cudaPos((size_t)bpos[0], (size_t)bpos[1], (size_t)bpos[2]);
    if (to_device) {
        prm.srcPtr = up; prm.srcPos = uo; prm.dstPtr = bp; prm.dstPos = bo;
    } else {
        prm.srcPtr = bp; prm.srcPos = bo; prm.dstPtr = up; prm.dstPos = uo;
    }
    prm.extent = make_cudaExtent((size_t)ext[0], (size_t)ext[1], (size_t)ext[2]);
    prm.kind = cudaMemcpyDefault;
    CUDA_TRY(cudaMemcpy3DAsync(&prm, g->stream));
    return HDARRAY_OK;
}

// A use of each device's region (Read, Reduce): exchange, then the bookkeeping.
int use_regions(HDArray *a, const Part &pt)
{
    grow_devices(a, pt.nparts);
    if (!g->host_only) {
        int jrc = join_write(a);
        if (jrc) return jrc;
    }
    std::vector<BoxSet> U(pt.nparts);
    for (int p = 0; p < pt.nparts; p++)
        if (!pt.box[p].empty()) U[p] = BoxSet{pt.box[p]};
    GState s = a->states[a->cur];
    std::vector<Move> moves;
    int rc = use_step(s, U, moves);
    if (rc) return rc;
    if (!g->host_only) {
        for (int p = 0; p < pt.nparts; p++) {
            if (!is_local(p)) continue;
            rc = ensure_buffer(a, p, pt.box[p]);
            if (rc) return rc;
        }
        std::vector<CopyTask> tasks;
        for (const Move &m : moves)
            if (is_local(m.src) && is_local(m.dst)) copy_tasks(a, a->buf[m.src], a->buf[m.dst], m.box, tasks);
        if (!tasks.empty()) {
            std::shared_ptr<DevMem> mem;
            std::vector<const char *> addr;
            rc = upload({{tasks.data(), tasks.size() * sizeof(CopyTask)}}, mem, addr);
            if (rc) return rc;
            LaunchRec L; L.kind = L_COPY; L.p0 = addr[0]; L.n0 = (int64_t)tasks.size();
            rc = issue_recorded(L);
            if (rc) return rc;
            CUDA_TRY(cudaStreamSynchronize(g->stream));  // the tables are freed on return
        }
    }
    rc = run_transport(a, moves);
    if (rc) return rc;
    for (const Move &m : moves) g->counters[1] += m.box.volume() * a->esize;
    a->cur = intern(a, std::move(s));
    a->last_moves = moves;
    return HDARRAY_OK;
}

int write_impl(HDArray *a, const void *uA, int part)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!a || !g->arrays.count(a)) return HDARRAY_ERR_INVAL;
    int rc = check_part_for(a, part);
    if (rc) return rc;
    if (g->recording) return HDARRAY_ERR_STATE;
    if (g->batching) {
        rc = flush_batch();
        if (rc) return rc;
    }
    const Part &pt = g->parts[part];
    grow_devices(a, pt.nparts);
    std::vector<BoxSet> D(pt.nparts);
    for (int p = 0; p < pt.nparts; p++)
        if (!pt.box[p].empty()) D[p] = BoxSet{pt.box[p]};
    GState s = a->states[a->cur];
    rc = def_step(s, D);
    if (rc) return rc;
    // From pinned host memory into buffers that already cover the regions: the copies run on the
    // library's copy stream after the library's last work on this array, so they overlap work on
    // other arrays; every later use of the array waits for them.
    bool async = false;
    if (!g->host_only && uA && g->async_write && !g->recording) {
        cudaPointerAttributes attr;
        async = cudaPointerGetAttributes(&attr, uA) == cudaSuccess && attr.type == cudaMemoryTypeHost;
        cudaGetLastError();
        for (int p = 0; async && p < pt.nparts; p++)
            if (!pt.box[p].empty() && is_local(p))
                async = a->buf[p].ptr && box_contains(a->buf[p].alloc, pt.box[p]);
    }
    if (async) {
        if (!g->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking));
        if (!a->write_ev) CUDA_TRY(cudaEventCreateWithFlags(&a->write_ev, cudaEventDisableTiming));
        if (!a->use_ev) CUDA_TRY(cudaEventCreateWithFlags(&a->use_ev, cudaEventDisableTiming));
        if (!a->track_use) {  // no use recorded yet: everything queued so far
            CUDA_TRY(cudaEventRecord(a->use_ev, g->stream));
            a->track_use = true;
        }
        CUDA_TRY(cudaStreamWaitEvent(g->copy_stream, a->use_ev, 0));
        if (a->write_pending) CUDA_TRY(cudaStreamWaitEvent(g->copy_stream, a->write_ev, 0));
        cudaStream_t lib_stream = g->stream;
        g->stream = g->copy_stream;  // memcpy_box queues on g->stream
        for (int p = 0; p < pt.nparts && !rc; p++) {
            if (pt.box[p].empty() || !is_local(p)) continue;
            rc = memcpy_box(a, a->buf[p], pt.box[p], const_cast<void *>(uA), true);
        }
        g->stream = lib_stream;
        if (rc) return rc;
        CUDA_TRY(cudaEventRecord(a->write_ev, g->copy_stream));
        a->write_pending = true;
    } else if (!g->host_only && uA) {
        rc = join_write(a);
        if (rc) return rc;
        for (int p = 0; p < pt.nparts; p++) {
            if (pt.box[p].empty() || !is_local(p)) continue;
            rc = ensure_buffer(a, p, pt.box[p]);
            if (rc) return rc;
            rc = memcpy_box(a, a->buf[p], pt.box[p], const_cast<void *>(uA), true);
            if (rc) return rc;
        }
        rc = note_use(a);
        if (rc) return rc;
    }
    a->cur = intern(a, std::move(s));
    a->version++;
    return HDARRAY_OK;
}

int read_impl(HDArray *a, void *uA, int part)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!a || !g->arrays.count(a)) return HDARRAY_ERR_INVAL;
    int rc = check_part_for(a, part);
    if (rc) return rc;
    if (g->recording) return HDARRAY_ERR_STATE;
    if (g->batching) {
        rc = flush_batch();
        if (rc) return rc;
    }
    const Part &pt = g->parts[part];
    rc = use_regions(a, pt);
    if (rc) return rc;
    if (!g->host_only && uA) {
        for (int p = 0; p < pt.nparts; p++) {
            if (pt.box[p].empty() || !is_local(p)) continue;
            rc = memcpy_box(a, a->buf[p], pt.box[p], uA, false);
            if (rc) return rc;
        }
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        return check_device_error();
    }
    return HDARRAY_OK;
}

// A kernel whose bounded device-side wait gave up leaves a non-zero error word; report it once.
int check_device_error()
{
    if (g->host_only || !g->err_word) return HDARRAY_OK;
    unsigned e = 0;
    if (cudaMemcpyAsync(&e, g->err_word, sizeof(e), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
        cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        return HDARRAY_ERR_CUDA;
    }
    if (e) {
        cudaMemsetAsync(g->err_word, 0, sizeof(unsigned), g->stream);
        return HDARRAY_ERR_TIMEOUT;
    }
    return HDARRAY_OK;
}

int ensure_reduce_scratch(int nblocks)
{
    if (g->red_blocks >= nblocks) return HDARRAY_OK;
    if (g->red_partials) cudaFree(g->red_partials);
    g->red_partials = nullptr;
    if (cudaMalloc(&g->red_partials, sizeof(double) * nblocks + 256) != cudaSuccess) {
        cudaGetLastError();
        g->red_blocks = 0;
        return HDARRAY_ERR_NOMEM;
    }
    g->red_blocks = nblocks;
    return HDARRAY_OK;
}

int reduce_impl(HDArray *a, double *res, int op, int part)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!a || !g->arrays.count(a) || !res || op < 0 || op > 3) return HDARRAY_ERR_INVAL;
    int rc = check_part_for(a, part);
    if (rc) return rc;
    if (g->recording) return HDARRAY_ERR_STATE;
    if (g->batching) {
        rc = flush_batch();
        if (rc) return rc;
    }
    const Part &pt = g->parts[part];
    for (int p = 0; p < pt.nparts; p++)
        for (int q = p + 1; q < pt.nparts; q++)
            if (box_overlaps(pt.box[p], pt.box[q])) return HDARRAY_ERR_INVAL;
    rc = use_regions(a, pt);
    if (rc) return rc;
    if (g->host_only) {
        *res = 0.0;
        return HDARRAY_OK;
    }
    const Ctx::SqSum &sq = g->sq_sum;
    if (op == HDARRAY_SUM && sq.R == a && sq.sum && sq.version == a->version && sq.boxes == pt.box &&
        a->last_moves.empty()) {
        // R is unchanged since the residual launch that defined it on exactly these boxes, and
        // that launch folded the sum of the values it stored: read it back
        CUDA_TRY(cudaMemcpyAsync(g->host_result, sq.sum, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        CUDA_TRY(cudaStreamSynchronize(g->stream));
        *res = *g->host_result;
        return check_device_error();
    }
    const auto key = std::make_tuple(a->uid, part, a->epoch);
    auto pit = g->red_plans.find(key);
    if (pit == g->red_plans.end()) {  // the task table of this (array, partition, buffers)
        std::vector<RedTask> tasks;
        for (int p = 0; p < pt.nparts; p++) {
            const Box &W = pt.box[p];
            if (W.empty() || !is_local(p)) continue;  // another rank folds its own devices
            const DevBuf &b = a->buf[p];
            View3 v = view_of(a, b, W);
            RedTask t;
            t.x = b.ptr + elem_off(b, W.lo) * a->esize;
            t.s_outer = v.s_outer;
            t.s_mid = v.s_mid;
            t.n_mid = (int32_t)v.n_mid;
            t.n_inner = (int32_t)v.n_inner;
            const int64_t rows = v.n_outer * v.n_mid;
            const int64_t per = std::max<int64_t>(1, 65536 / std::max<int64_t>(1, v.n_inner));
            for (int64_t r = 0; r < rows; r += per) {
                t.row_begin = (int32_t)r;
                t.row_end = (int32_t)std::min(rows, r + per);
                tasks.push_back(t);
            }
        }
        Ctx::RedPlan rp;
        rp.ntasks = (int)tasks.size();
        rp.nblocks = (int)std::min<size_t>(tasks.size(), (size_t)2 * g->nsm);
        if (!tasks.empty()) {
            std::vector<const char *> addr;
            rc = upload({{tasks.data(), tasks.size() * sizeof(RedTask)}}, rp.mem, addr);
            if (rc) return rc;
        }
        if (g->red_plans.size() >= 256) g->red_plans.clear();
        pit = g->red_plans.emplace(key, std::move(rp)).first;
    }
    const Ctx::RedPlan &rp = pit->second;
    const double ident[4] = {0.0, 1.0, -__builtin_inf(), __builtin_inf()};
    if (rp.ntasks == 0) {
        *res = ident[op];
        return HDARRAY_OK;
    }
    rc = ensure_reduce_scratch(rp.nblocks);
    if (rc) return rc;
    CUDA_TRY(launch_reduce(a->dtype, op, (const RedTask *)rp.mem->ptr, rp.ntasks, rp.nblocks,
                           g->red_partials, g->red_counter, g->red_result, g->stream));
    g->counters[0]++;
    CUDA_TRY(cudaMemcpyAsync(g->host_result, g->red_result, sizeof(double), cudaMemcpyDeviceToHost,
                             g->stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    *res = *g->host_result;
    return check_device_error();
}

// ------------------------------------------------------------------------------------------
// Partitions
// ------------------------------------------------------------------------------------------

void split_even(int64_t a, int64_t b, int P, int p, int64_t *lo, int64_t *hi)
{
    const int64_t n = b - a, q = n / P, m = n % P;
    *lo = a + p * q + std::min<int64_t>(p, m);
    *hi = *lo + q + (p < m ? 1 : 0);
}

int make_partition(int type, int nparts, int dim, const int64_t *sizes, const int64_t *lo, const int64_t *hi)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (dim < 1 || dim > 3 || !sizes || !lo || !hi) return HDARRAY_ERR_INVAL;
    if (nparts <= 0) nparts = g->ndev;
    if (nparts > 32767) return HDARRAY_ERR_INVAL;
    Part pt;
    pt.dim = dim;
    pt.nparts = nparts;
    Box region = make_box(0, 0, 0, 1, 1, 1);
    for (int d = 0; d < dim; d++) {
        pt.n[d] = sizes[d];
        if (sizes[d] < 1 || lo[d] < 0 || hi[d] > sizes[d] || lo[d] > hi[d]) return HDARRAY_ERR_RANGE;
        region.lo[d] = lo[d];
        region.hi[d] = hi[d];
    }
    if ((type == HDARRAY_COL || type == HDARRAY_BLOCK) && dim < 2) return HDARRAY_ERR_INVAL;
    int Pr = 1, Pc = nparts;
    if (type == HDARRAY_BLOCK) {
        for (int d = 1; d * d <= nparts; d++)
            if (nparts % d == 0) Pr = d;
        Pc = nparts / Pr;
    }
    for (int p = 0; p < nparts; p++) {
        Box b = region;
        if (type == HDARRAY_ROW) split_even(region.lo[0], region.hi[0], nparts, p, &b.lo[0], &b.hi[0]);
        else if (type == HDARRAY_COL) split_even(region.lo[1], region.hi[1], nparts, p, &b.lo[1], &b.hi[1]);
        else if (type == HDARRAY_BLOCK) {
            split_even(region.lo[0], region.hi[0], Pr, p / Pc, &b.lo[0], &b.hi[0]);
            split_even(region.lo[1], region.hi[1], Pc, p % Pc, &b.lo[1], &b.hi[1]);
        } else {
            return HDARRAY_ERR_INVAL;
        }
        pt.box.push_back(b);
    }
    g->parts.push_back(pt);
    return (int)g->parts.size() - 1;
}

int set_abs(const char *kname, int part, HDArray *a, int dev, const std::vector<Box> &boxes, bool use)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!kname || !a || !g->arrays.count(a) || dev < 0 || dev > 32767) return HDARRAY_ERR_INVAL;
    if (part < 0 || part >= (int)g->parts.size()) return HDARRAY_ERR_INVAL;
    Ctx::AbsSpec &s = g->abs[std::make_tuple(std::string(kname), part, a->uid)];
    auto &m = use ? s.use : s.def;
    auto &v = m[dev];
    v.insert(v.end(), boxes.begin(), boxes.end());
    if (use) s.has_use = true;
    else s.has_def = true;
    s.version = ++g->abs_version;
    return HDARRAY_OK;
}

int abs_box(const char *kname, int part, HDArray *a, int dev, int dim, const int64_t *lo,
            const int64_t *hi, bool use)
{
    if (!g || !a || !lo || !hi || dim != a->dim) return HDARRAY_ERR_INVAL;
    Box b = make_box(0, 0, 0, 1, 1, 1);
    for (int d = 0; d < dim; d++) {
        b.lo[d] = lo[d];
        b.hi[d] = hi[d];
        if (lo[d] < 0 || hi[d] > a->n[d]) return HDARRAY_ERR_RANGE;
    }
    return set_abs(kname, part, a, dev, {b}, use);
}

int abs_trap(const char *kname, int part, HDArray *a, int dev, const int64_t *c, bool use)
{
    if (!g || !a || !c || a->dim != 2) return HDARRAY_ERR_INVAL;
    BoxSet s;
    if (!trapezoid_boxes(c, &s)) return HDARRAY_ERR_INVAL;
    for (const Box &b : s)
        if (b.lo[0] < 0 || b.hi[0] > a->n[0] || b.lo[1] < 0 || b.hi[1] > a->n[1]) return HDARRAY_ERR_RANGE;
    return set_abs(kname, part, a, dev, std::vector<Box>(s.begin(), s.end()), use);
}

void free_array_buffers(HDArray *a)
{
    if (a->write_ev) cudaEventSynchronize(a->write_ev);
    for (DevBuf &b : a->buf)
        if (b.ptr) dev_free(b.ptr);
    a->buf.clear();
    if (a->write_ev) cudaEventDestroy(a->write_ev);
    if (a->use_ev) cudaEventDestroy(a->use_ev);
    a->write_ev = a->use_ev = nullptr;
    a->write_pending = a->track_use = false;
}

void drop_plans_of(HDArray *a)
{
    for (auto it = g->memo.begin(); it != g->memo.end();) {
        bool hit = false;
        for (HDArray *x : it->second->args) hit = hit || x == a;
        if (hit) it = g->memo.erase(it);
        else ++it;
    }
    g->batch_cache.clear();
}

int init_impl(int ndev, unsigned flags)
{
    if (g && g->inited) return HDARRAY_OK;
    if (ndev < 1) return HDARRAY_ERR_INVAL;
    g = new Ctx();
    g->ndev = ndev;
    g->host_only = (flags & HDARRAY_INIT_HOST_ONLY) != 0;
    register_builtins(*g);
    if (!g->host_only) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            g = nullptr;
            return HDARRAY_ERR_CUDA;
        }
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) g->nsm = prop.multiProcessorCount;
        if (cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete g;
            g = nullptr;
            return HDARRAY_ERR_CUDA;
        }
        g->stream = g->own_stream;
        void *p = nullptr;
        if (cudaMalloc(&p, 256) != cudaSuccess) {
            cudaGetLastError();
            return HDARRAY_ERR_NOMEM;
        }
        g->red_counter = (unsigned *)p;
        g->err_word = (unsigned *)((char *)p + 64);
        g->red_result = (double *)((char *)p + 128);
        cudaMemset(p, 0, 256);
        if (cudaMallocHost(&g->host_result, sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return HDARRAY_ERR_NOMEM;
        }
        const char *tr = getenv("HDARRAY_TILE_ROWS");
        if (tr && atoi(tr) > 0) g->tile_rows = atoi(tr);
        const char *wc = getenv("HDARRAY_WARPS_PER_CTA");
        if (wc && atoi(wc) > 0 && atoi(wc) <= 8) g->warps_per_cta = atoi(wc);
        const char *vv = getenv("HDARRAY_JACOBI_VARIANT");
        if (vv && atoi(vv) >= 0 && atoi(vv) <= 5) g->variant = atoi(vv);
        const char *lr = getenv("HDARRAY_LATE_RECEIVE");
        if (lr && (atoi(lr) == 0 || atoi(lr) == 1)) g->late = atoi(lr);
        const char *sn = getenv("HDARRAY_SNAKE");
        if (sn && (atoi(sn) == 0 || atoi(sn) == 1)) g->snake = atoi(sn);
        const char *ra = getenv("HDARRAY_ROW_ALIGN");
        if (ra && atoi(ra) >= 16 && atoi(ra) <= 1024 && (atoi(ra) & (atoi(ra) - 1)) == 0) g->row_align = atoi(ra);
        const char *b2 = getenv("HDARRAY_BAND2");
        if (b2 && atoi(b2) > 0) g->band2 = atoi(b2);
        const char *at = getenv("HDARRAY_AUTOTUNE");
        g->autotune = at && atoi(at) != 0;
        const char *aw = getenv("HDARRAY_ASYNC_WRITE");
        if (aw) g->async_write = atoi(aw) != 0;
        const char *fx = getenv("HDARRAY_FUSE_EXCHANGE");
        if (fx) g->fuse = atoi(fx) != 0;
        const char *v3 = getenv("HDARRAY_STENCIL3D_VARIANT");
        if (v3 && atoi(v3) >= 0 && atoi(v3) <= 3) g->variant3 = atoi(v3);
        const char *tz = getenv("HDARRAY_TILE_Z");
        if (tz && atoi(tz) > 0) g->tile_z = atoi(tz);
        const char *sl = getenv("HDARRAY_SPIN_LIMIT");
        if (sl && *sl) g->spin_limit = (unsigned)strtoul(sl, nullptr, 10);
        const char *b3 = getenv("HDARRAY_BAND3");
        if (b3 && atoi(b3) > 0) g->band3 = atoi(b3);
        const char *c3 = getenv("HDARRAY_CTA3");
        if (c3 && (atoi(c3) == 256 || atoi(c3) == 512)) g->cta3 = atoi(c3);
    }
    g->inited = true;
    return HDARRAY_OK;
}

}  // namespace

namespace hda {

DevMem::~DevMem()
{
    if (ptr) dev_free(ptr);
}

namespace {
struct AllocHooks {
    HDArrayAlloc_t alloc = nullptr;
    HDArrayFree_t free_fn = nullptr;
    void *user = nullptr;
};
AllocHooks g_hooks;
std::unordered_map<void *, AllocHooks> g_custom;  // allocations made through a caller's allocator
int g_user_rc = 0;                                // a user launcher's last failure code
}  // namespace

int dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (g_hooks.alloc) {
        void *q = g_hooks.alloc(bytes, g_hooks.user);
        if (!q) return HDARRAY_ERR_NOMEM;
        if ((uintptr_t)q % 256 != 0) {  // the buffers' row phase and the bulk copies need it
            g_hooks.free_fn(q, g_hooks.user);
            return HDARRAY_ERR_INVAL;
        }
        g_custom[q] = g_hooks;
        *p = q;
        return HDARRAY_OK;
    }
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return HDARRAY_ERR_NOMEM;
    }
    return HDARRAY_OK;
}

void dev_free(void *p)
{
    if (!p) return;
    auto it = g_custom.find(p);
    if (it != g_custom.end()) {
        const AllocHooks h = it->second;
        g_custom.erase(it);
        // cudaFree waits for the device; a caching allocator may hand the memory to other work at
        // once, so wait for every queued use of it first
        cudaDeviceSynchronize();
        h.free_fn(p, h.user);
        return;
    }
    cudaFree(p);
}

int set_allocator(HDArrayAlloc_t alloc, HDArrayFree_t free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return HDARRAY_ERR_INVAL;
    g_hooks.alloc = alloc;
    g_hooks.free_fn = free_fn;
    g_hooks.user = user;
    return HDARRAY_OK;
}

int user_launch_rc() { return g_user_rc; }

cudaError_t issue(const LaunchRec &L, cudaStream_t s)
{
    switch (L.kind) {
    case L_COPY: return launch_copy((const CopyTask *)L.p0, (int)L.n0, s);
    case L_JACOBI2D:
        if (L.n2 == 5)
            return launch_jacobi2d_tma(0, L.dtype, (const StenPart2D *)L.p0, (const StenTile2D *)L.p1, (int)L.n0,
                                       (const Seg *)L.p2, (size_t)L.n3, s, L.p3, nullptr, g->err_word, g->spin_limit,
                                       (int)L.n1);
        return launch_jacobi2d(L.dtype, (const StenPart2D *)L.p0, (const StenTile2D *)L.p1, (int)L.n0,
                               (const Seg *)L.p2, (int)L.n1, (int)L.n2, (size_t)L.n3, s);
    case L_STENCIL3D:
        return launch_stencil3d(L.dtype, (const StenPart3D *)L.p0, (const StenTile3D *)L.p1, (int)L.n0,
                                (const Seg *)L.p2, (int)L.n1, (int)L.n2, (size_t)L.n3, s, L.p3, g->err_word,
                                g->spin_limit);
    case L_SQDIFF: {
        char *red = (char *)const_cast<void *>(L.p1);
        unsigned *counter = red ? (unsigned *)(red + red_counter_offset(L.n1)) : nullptr;
        double *sum = red ? (double *)(red + red_counter_offset(L.n1) + 128) : nullptr;
        return launch_sqdiff(L.dtype, (const PwTask *)L.p0, (int)L.n0, (int)L.n1, (double *)red, counter, sum, s);
    }
    case L_GEMM64:
        return launch_gemm_f64((const GemmPart *)L.p0, (int)L.n0, (int)L.n1, (int)L.n2, L.f0, L.f1, s);
    case L_GEMM_TC:
        return launch_gemm_tc((const TcPart *)L.p0, (const TcTile *)L.p1, (int)L.n0, (float)L.f0, (float)L.f1,
                              (unsigned *)L.p2, s);
    case L_SPLIT: return launch_split_panels((const SplitJob *)L.p0, (int)L.n0, (int)L.n1, s);
    case L_USER: {
        const KernelDef *kd = (const KernelDef *)L.p2;
        const int rc = kd->launcher((const HDArrayWork_t *)L.p0, (int)L.n0, (const double *)L.p1, (int)L.n1,
                                    (void *)s, kd->user);
        if (rc == 0) return cudaSuccess;
        g_user_rc = rc < 0 ? rc : HDARRAY_ERR_CUDA;
        return cudaErrorUnknown;
    }
    case L_COLMEAN: return launch_colmean(L.dtype, (const CovTask *)L.p0, (int)L.n0, (int)L.n2, s);
    case L_CENTER: return launch_center(L.dtype, (const CovTask *)L.p0, (int)L.n0, (int)L.n1, s);
    case L_SYMM: return launch_symmetrize(L.dtype, (const CovTask *)L.p0, (int)L.n0, (int)L.n1, (int)L.n2, s);
    case L_CONV2D:
        if (L.n2 == 5)
            return launch_jacobi2d_tma(1, L.dtype, (const StenPart2D *)L.p0, (const StenTile2D *)L.p1, (int)L.n0,
                                       (const Seg *)L.p2, (size_t)L.n3, s, L.p3, (const double *)L.p4, g->err_word,
                                       g->spin_limit, (int)L.n1);
        return launch_stencil2d_cta(1, L.dtype, (const StenPart2D *)L.p0, (const StenTile2D *)L.p1, (int)L.n0,
                                    (const Seg *)L.p2, (const double *)L.p3, (size_t)L.n3, s);
    case L_FLAT2D:
        return launch_jacobi2d_flat(L.dtype, (const StenPart2D *)L.p0, (const StenTile2D *)L.p1, (int)L.n0,
                                    (const Seg *)L.p2, (size_t)L.n1, s);
    case L_FLAT3D:
        return launch_stencil3d_flat(L.dtype, (const StenPart3D *)L.p0, (const StenTile3D *)L.p1, (int)L.n0,
                                     (const Seg *)L.p2, (size_t)L.n1, s);
    case L_GEMM_PANEL:
        return launch_gemm_panels((const PanelPart *)L.p0, (const TcTile *)L.p1, (int)L.n0, (float)L.f0,
                                  (float)L.f1, (unsigned *)L.p2, (unsigned)L.n3, (int)L.n1, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hda

// ==========================================================================================
// C ABI
// ==========================================================================================

extern "C" {

int HDArrayInitEx(int ndev, unsigned flags) { return init_impl(ndev, flags); }

int HDArrayInit(int argc, char *argv[], const char *kpath, const char *dpath)
{
    (void)argc;
    (void)argv;
    (void)kpath;
    int ndev = 1;
    const char *env = getenv("HDARRAY_NDEV");
    if (env && atoi(env) > 0) ndev = atoi(env);
    if (dpath) {
        FILE *f = fopen(dpath, "r");
        if (!f) return HDARRAY_ERR_INVAL;
        int n = 0;
        if (fscanf(f, "%d", &n) != 1 || n < 1) {
            fclose(f);
            return HDARRAY_ERR_INVAL;
        }
        fclose(f);
        ndev = n;
    }
    int rc = init_impl(ndev, 0);
    return rc < 0 ? rc : 0;
}

void HDArrayExit(void)
{
    if (!g) return;
    if (g->copy_stream) cudaStreamSynchronize(g->copy_stream);
    if (g->stream) cudaStreamSynchronize(g->stream);
    for (auto &kv : g->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    g->graphs.clear();
    g->sq_sum = Ctx::SqSum();
    g->red_plans.clear();
    g->memo.clear();
    g->batch.clear();
    g->batch_cache.clear();
    g->rec_refs.clear();
    g->rec_mems.clear();
    for (HDArray *a : g->arrays) {
        free_array_buffers(a);
        delete a;
    }
    g->arrays.clear();
    if (g->red_partials) cudaFree(g->red_partials);
    if (g->red_counter) cudaFree(g->red_counter);
    if (g->host_result) cudaFreeHost(g->host_result);
    if (g->own_stream) cudaStreamDestroy(g->own_stream);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    delete g;
    g = nullptr;
}

void HDArrayShowDeviceInfo(int devID)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, devID) != cudaSuccess) {
        cudaGetLastError();
        printf("HDArray device %d: no CUDA device\n", devID);
        return;
    }
    printf("HDArray device %d: %s, sm_%d%d, %d SMs, %.1f GiB, %d logical devices\n", devID, prop.name,
           prop.major, prop.minor, prop.multiProcessorCount, prop.totalGlobalMem / 1073741824.0,
           g ? g->ndev : 0);
}

HDArray_t *HDArrayCreatev(const char *sym, const char *type, void *uA, int dim, const int64_t *sizes)
{
    (void)uA;
    if (!g || !g->inited) {
        set_err(HDARRAY_ERR_STATE);
        return nullptr;
    }
    int esize = 0;
    int dt = dtype_of(type, &esize);
    if (dt < 0 || dim < 1 || dim > 3 || !sizes) {
        set_err(HDARRAY_ERR_INVAL);
        return nullptr;
    }
    HDArray *a = new HDArray();
    a->sym = sym ? sym : "";
    a->dtype = dt;
    a->esize = esize;
    a->dim = dim;
    for (int d = 0; d < dim; d++) {
        if (sizes[d] < 1 || sizes[d] > (int64_t)1 << 31) {
            delete a;
            set_err(HDARRAY_ERR_INVAL);
            return nullptr;
        }
        a->n[d] = sizes[d];
    }
    a->uid = g->next_uid++;
    a->states.push_back(GState{});
    a->states[0].hash = hash_state(a->states[0]);
    a->cur = 0;
    g->arrays.insert(a);
    return a;
}

HDArray_t *HDArrayCreate(const char *sym, const char *type, void *uA, int dim, ...)
{
    if (dim < 1 || dim > 3) {
        set_err(HDARRAY_ERR_INVAL);
        return nullptr;
    }
    int64_t sizes[3];
    va_list ap;
    va_start(ap, dim);
    for (int d = 0; d < dim; d++) sizes[d] = va_arg(ap, int);
    va_end(ap);
    return HDArrayCreatev(sym, type, uA, dim, sizes);
}

int HDArrayFree(HDArray_t *hA)
{
    if (!g || !hA || !g->arrays.count(hA)) return HDARRAY_ERR_INVAL;
    if (g->copy_stream) cudaStreamSynchronize(g->copy_stream);
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (g->sq_sum.R == hA) g->sq_sum = Ctx::SqSum();
    for (auto it = g->red_plans.begin(); it != g->red_plans.end();) {
        if (std::get<0>(it->first) == hA->uid) it = g->red_plans.erase(it);
        else ++it;
    }
    drop_plans_of(hA);
    for (auto it = g->abs.begin(); it != g->abs.end();) {
        if (std::get<2>(it->first) == hA->uid) it = g->abs.erase(it);
        else ++it;
    }
    free_array_buffers(hA);
    g->arrays.erase(hA);
    delete hA;
    return HDARRAY_OK;
}

int HDArrayPartitionv(PART_T type, int nparts, int dim, const int64_t *sizes, const int64_t *lo,
                      const int64_t *hi)
{
    return make_partition((int)type, nparts, dim, sizes, lo, hi);
}

int HDArrayPartition(PART_T type, int dim, ...)
{
    if (dim < 1 || dim > 3) return set_err(HDARRAY_ERR_INVAL);
    int64_t s[3], lo[3], hi[3];
    va_list ap;
    va_start(ap, dim);
    for (int d = 0; d < dim; d++) s[d] = va_arg(ap, int);
    for (int d = 0; d < dim; d++) lo[d] = va_arg(ap, int);
    for (int d = 0; d < dim; d++) hi[d] = va_arg(ap, int);
    va_end(ap);
    int rc = make_partition((int)type, 0, dim, s, lo, hi);
    if (rc < 0) set_err(rc);
    return rc;
}

int HDArrayPartitionManual(int dim, const int64_t *sizes, int nparts, const int64_t *lo, const int64_t *hi)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (dim < 1 || dim > 3 || nparts < 1 || nparts > 32767 || !sizes || !lo || !hi) return HDARRAY_ERR_INVAL;
    Part pt;
    pt.dim = dim;
    pt.nparts = nparts;
    for (int d = 0; d < dim; d++) {
        if (sizes[d] < 1) return HDARRAY_ERR_INVAL;
        pt.n[d] = sizes[d];
    }
    for (int p = 0; p < nparts; p++) {
        Box b = make_box(0, 0, 0, 1, 1, 1);
        for (int d = 0; d < dim; d++) {
            b.lo[d] = lo[p * dim + d];
            b.hi[d] = hi[p * dim + d];
            if (b.lo[d] < 0 || b.hi[d] > sizes[d]) return HDARRAY_ERR_RANGE;
        }
        if (b.empty()) b = make_box(0, 0, 0, 0, 0, 0);
        pt.box.push_back(b);
    }
    g->parts.push_back(pt);
    return (int)g->parts.size() - 1;
}

int HDArrayApplyKernelv(const char *kName, int partID, int narr, HDArray_t *const *arrs, int nscal,
                        const double *scal)
{
    if (narr < 0 || (narr > 0 && !arrs) || nscal < 0 || (nscal > 0 && !scal)) return HDARRAY_ERR_INVAL;
    std::vector<HDArray *> a(arrs, arrs + narr);
    std::vector<double> s(scal, scal + nscal);
    int rc = apply(kName, partID, a, s);
    if (rc) set_err(rc);
    return rc;
}

void HDArrayApplyKernel(const char *kName, int partID, ...)
{
    if (!g || !g->inited || !kName) {
        set_err(HDARRAY_ERR_STATE);
        return;
    }
    auto it = g->kernels.find(kName);
    if (it == g->kernels.end()) {
        set_err(HDARRAY_ERR_INVAL);
        return;
    }
    const KernelDef &k = it->second;
    std::vector<HDArray *> a;
    std::vector<double> s;
    va_list ap;
    va_start(ap, partID);
    for (int i = 0; i < k.narr; i++) a.push_back(va_arg(ap, HDArray *));
    for (int i = 0; i < k.nscal_f; i++) s.push_back(va_arg(ap, double));
    for (int i = 0; i < k.nscal_i; i++) s.push_back((double)va_arg(ap, int));
    va_end(ap);
    int rc = apply(kName, partID, a, s);
    if (rc) set_err(rc);
}

int HDArrayWritev(HDArray_t *hA, const void *uA, int partID)
{
    int rc = write_impl(hA, uA, partID);
    if (rc) set_err(rc);
    return rc;
}

void HDArrayWrite(HDArray_t *hA, void *uA, int partID) { HDArrayWritev(hA, uA, partID); }

int HDArrayReadv(HDArray_t *hA, void *uA, int partID)
{
    int rc = read_impl(hA, uA, partID);
    if (rc) set_err(rc);
    return rc;
}

void HDArrayRead(HDArray_t *hA, void *uA, int partID) { HDArrayReadv(hA, uA, partID); }

int HDArrayReduceD(HDArray_t *hA, double *res, REDUCE_OP op, int partID)
{
    int rc = reduce_impl(hA, res, (int)op, partID);
    if (rc) set_err(rc);
    return rc;
}

int HDArrayReducev(HDArray_t *hA, void *res, REDUCE_OP op, int partID)
{
    if (!res) return set_err(HDARRAY_ERR_INVAL);
    double d = 0.0;
    int rc = reduce_impl(hA, &d, (int)op, partID);
    if (rc) return set_err(rc);
    if (hA->dtype == DT_F64) {
        *(double *)res = d;
    } else if (hA->dtype == DT_F32) {
        *(float *)res = (float)d;
    } else {  // bfloat16, round to nearest even
        float f = (float)d;
        uint32_t u;
        memcpy(&u, &f, 4);
        uint32_t up = u >> 16, low = u & 0xffffu;
        if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) up |= 0x40;
        else if (low > 0x8000u || (low == 0x8000u && (up & 1u))) up += 1;
        *(uint16_t *)res = (uint16_t)up;
    }
    return HDARRAY_OK;
}

void HDArrayReduce(HDArray_t *hA, void *res, REDUCE_OP op, int partID) { HDArrayReducev(hA, res, op, partID); }

int HDArraySetAbsoluteUsev(const char *kName, int partID, HDArray_t *hA, int devID, int dim,
                           const int64_t *lo, const int64_t *hi)
{
    int rc = abs_box(kName, partID, hA, devID, dim, lo, hi, true);
    if (rc) set_err(rc);
    return rc;
}

int HDArraySetAbsoluteDefv(const char *kName, int partID, HDArray_t *hA, int devID, int dim,
                           const int64_t *lo, const int64_t *hi)
{
    int rc = abs_box(kName, partID, hA, devID, dim, lo, hi, false);
    if (rc) set_err(rc);
    return rc;
}

static void abs_varargs(const char *kName, int partID, HDArray_t *hA, int devID, int dim, va_list ap, bool use)
{
    if (dim < 1 || dim > 3) {
        set_err(HDARRAY_ERR_INVAL);
        return;
    }
    int64_t lo[3], hi[3];
    for (int d = 0; d < dim; d++) lo[d] = va_arg(ap, int);
    for (int d = 0; d < dim; d++) hi[d] = va_arg(ap, int);
    int rc = abs_box(kName, partID, hA, devID, dim, lo, hi, use);
    if (rc) set_err(rc);
}

void HDArraySetAbsoluteUse(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...)
{
    va_list ap;
    va_start(ap, dim);
    abs_varargs(kName, partID, hA, devID, dim, ap, true);
    va_end(ap);
}

void HDArraySetAbsoluteDef(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...)
{
    va_list ap;
    va_start(ap, dim);
    abs_varargs(kName, partID, hA, devID, dim, ap, false);
    va_end(ap);
}

int HDArraySetTrapezoidUsev(const char *kName, int partID, HDArray_t *hA, int devID, const int64_t *corners)
{
    int rc = abs_trap(kName, partID, hA, devID, corners, true);
    if (rc) set_err(rc);
    return rc;
}

int HDArraySetTrapezoidDefv(const char *kName, int partID, HDArray_t *hA, int devID, const int64_t *corners)
{
    int rc = abs_trap(kName, partID, hA, devID, corners, false);
    if (rc) set_err(rc);
    return rc;
}

static void trap_varargs(const char *kName, int partID, HDArray_t *hA, int devID, int dim, va_list ap, bool use)
{
    if (dim != 2) {
        set_err(HDARRAY_ERR_INVAL);
        return;
    }
    int64_t c[8];
    for (int i = 0; i < 8; i++) c[i] = va_arg(ap, int);
    int rc = abs_trap(kName, partID, hA, devID, c, use);
    if (rc) set_err(rc);
}

void HDArraySetTrapezoidUse(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...)
{
    va_list ap;
    va_start(ap, dim);
    trap_varargs(kName, partID, hA, devID, dim, ap, true);
    va_end(ap);
}

void HDArraySetTrapezoidDef(const char *kName, int partID, HDArray_t *hA, int devID, int dim, ...)
{
    va_list ap;
    va_start(ap, dim);
    trap_varargs(kName, partID, hA, devID, dim, ap, false);
    va_end(ap);
}

static int set_offsets(const char *kName, int argIndex, int noff, const int32_t *offs, bool use)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!kName || noff < 0 || (noff > 0 && !offs)) return HDARRAY_ERR_INVAL;
    auto it = g->kernels.find(kName);
    if (it == g->kernels.end()) return HDARRAY_ERR_INVAL;
    KernelDef &k = it->second;
    if (argIndex < 0 || argIndex >= k.narr) return HDARRAY_ERR_INVAL;
    std::vector<Offset> v;
    for (int i = 0; i < noff; i++) v.push_back(Offset{{offs[3 * i], offs[3 * i + 1], offs[3 * i + 2]}});
    (use ? k.use : k.def)[argIndex] = v;
    k.version++;
    return HDARRAY_OK;
}

int HDArrayRegisterKernel(const char *kName, int narr, int nscal, int spaceArg, HDArrayLauncher_t launcher,
                          void *user)
{
    if (!g || !g->inited) return set_err(HDARRAY_ERR_STATE);
    if (!kName || !*kName || !launcher || narr < 1 || narr > HDARRAY_MAX_KERNEL_ARRAYS || nscal < 0 ||
        spaceArg < 0 || spaceArg >= narr)
        return set_err(HDARRAY_ERR_INVAL);
    auto it = g->kernels.find(kName);
    if (it != g->kernels.end() && it->second.kind != K_USER) return set_err(HDARRAY_ERR_INVAL);
    KernelDef k;
    k.name = kName;
    k.kind = K_USER;
    k.narr = narr;
    k.nscal_f = nscal;
    k.space = spaceArg;
    k.use.assign(narr, {});
    k.def.assign(narr, {});
    k.launcher = launcher;
    k.user = user;
    if (it != g->kernels.end()) k.version = it->second.version + 1;  // plans of the old one are stale
    g->kernels[kName] = k;
    return HDARRAY_OK;
}

int HDArraySetAllocator(HDArrayAlloc_t alloc, HDArrayFree_t free_fn, void *user)
{
    return set_err(set_allocator(alloc, free_fn, user));
}

int HDArraySetOffsetUse(const char *kName, int argIndex, int noff, const int32_t *offs)
{
    return set_offsets(kName, argIndex, noff, offs, true);
}

int HDArraySetOffsetDef(const char *kName, int argIndex, int noff, const int32_t *offs)
{
    return set_offsets(kName, argIndex, noff, offs, false);
}

int HDArrayNumDevices(void) { return g ? g->ndev : 0; }

int HDArraySetStream(void *stream)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (g->recording || g->batching) return HDARRAY_ERR_STATE;
    g->stream = stream ? (cudaStream_t)stream : g->own_stream;
    return HDARRAY_OK;
}

int HDArraySetMode(int mode)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (mode != HDARRAY_MODE_FUSED && mode != HDARRAY_MODE_PLAIN) return HDARRAY_ERR_INVAL;
    if (g->recording || g->batching) return HDARRAY_ERR_STATE;
    if (mode != g->mode) {
        g->mode = mode;
        for (auto &kv : g->memo) kv.second->compiled_sig.clear();
        g->batch_cache.clear();
    }
    return HDARRAY_OK;
}

int HDArraySetGemmSplit(int parts)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (parts != HDARRAY_GEMM_BF16X3 && parts != HDARRAY_GEMM_BF16X6) return HDARRAY_ERR_INVAL;
    if (g->recording || g->batching) return HDARRAY_ERR_STATE;
    if (parts != g->gemm_parts) {
        g->gemm_parts = parts;
        for (auto &kv : g->memo) kv.second->compiled_sig.clear();  // recompiled on their next use
        g->batch_cache.clear();
    }
    return HDARRAY_OK;
}

int HDArraySetAutotune(int on)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    g->autotune = on != 0;
    return HDARRAY_OK;
}

int HDArrayBatchBegin(void)
{
    if (!g || !g->inited || g->batching) return HDARRAY_ERR_STATE;
    g->batching = true;
    g->batch_used.clear();
    g->batch_defined.clear();
    return HDARRAY_OK;
}

int HDArrayBatchEnd(void)
{
    if (!g || !g->inited || !g->batching) return HDARRAY_ERR_STATE;
    g->batching = false;
    g->batch_used.clear();
    g->batch_defined.clear();
    int rc = flush_batch();
    if (rc) set_err(rc);
    return rc;
}

int HDArrayGraphBegin(void)
{
    if (!g || !g->inited || g->recording || g->batching) return HDARRAY_ERR_STATE;
    if (g->host_only) return HDARRAY_ERR_UNSUPPORTED;
    g->recording = true;
    g->rec_invalid = false;
    g->rec.clear();
    g->rec_refs.clear();
    g->rec_mems.clear();
    g->rec_pre.clear();
    g->rec_defined.clear();
    return HDARRAY_OK;
}

int HDArrayGraphEnd(int *graphID)
{
    if (!g || !g->inited || !g->recording || !graphID) return HDARRAY_ERR_STATE;
    g->recording = false;
    if (g->rec_invalid) return set_err(HDARRAY_ERR_STATE);
    GraphRec gr;
    for (auto &kv : g->rec_pre) {
        HDArray *a = kv.first;
        if (a->generation != kv.second.second) return set_err(HDARRAY_ERR_STATE);
        gr.arrays.push_back({a, a->generation, a->epoch, kv.second.first, a->cur});
    }
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    for (const LaunchRec &L : g->rec) {
        cudaError_t e = issue(L, g->stream);
        if (e != cudaSuccess) {
            cudaGraph_t dummy;
            cudaStreamEndCapture(g->stream, &dummy);
            if (dummy) cudaGraphDestroy(dummy);
            return set_err(HDARRAY_ERR_CUDA);
        }
    }
    CUDA_TRY(cudaStreamEndCapture(g->stream, &gr.graph));
    CUDA_TRY(cudaGraphInstantiate(&gr.exec, gr.graph, 0));
    gr.refs = g->rec_refs;
    gr.mems = g->rec_mems;
    gr.defined.assign(g->rec_defined.begin(), g->rec_defined.end());
    gr.nkernels = (int64_t)g->rec.size();
    g->rec.clear();
    g->rec_refs.clear();
    g->rec_mems.clear();
    const int id = g->next_graph++;
    g->graphs[id] = std::move(gr);
    *graphID = id;
    return HDARRAY_OK;
}

int HDArrayGraphLaunch(int graphID, int nrep)
{
    if (!g || !g->inited || g->recording || g->batching) return HDARRAY_ERR_STATE;
    auto it = g->graphs.find(graphID);
    if (it == g->graphs.end() || nrep < 0) return HDARRAY_ERR_INVAL;
    GraphRec &gr = it->second;
    for (auto &ai : gr.arrays) {
        if (!g->arrays.count(ai.a)) return set_err(HDARRAY_ERR_STATE);
        if (ai.a->generation != ai.generation || ai.a->epoch != ai.epoch || ai.a->cur != ai.pre)
            return set_err(HDARRAY_ERR_STATE);
        if (nrep > 1 && ai.pre != ai.post) return set_err(HDARRAY_ERR_STATE);
    }
    for (auto &ai : gr.arrays) {
        const int rc = join_write(ai.a);
        if (rc) return set_err(rc);
    }
    for (int r = 0; r < nrep; r++) CUDA_TRY(cudaGraphLaunch(gr.exec, g->stream));
    if (nrep > 0) {
        for (auto &ai : gr.arrays) {
            ai.a->cur = ai.post;
            const int rc = note_use(ai.a);
            if (rc) return set_err(rc);
        }
        for (HDArray *a : gr.defined) a->version += (uint64_t)nrep;  // their contents changed
    }
    g->counters[0] += gr.nkernels * nrep;
    g->counters[4] += nrep;
    return HDARRAY_OK;
}

int HDArrayGraphDestroy(int graphID)
{
    if (!g) return HDARRAY_ERR_STATE;
    auto it = g->graphs.find(graphID);
    if (it == g->graphs.end()) return HDARRAY_ERR_INVAL;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (it->second.exec) cudaGraphExecDestroy(it->second.exec);
    if (it->second.graph) cudaGraphDestroy(it->second.graph);
    g->graphs.erase(it);
    return HDARRAY_OK;
}

int HDArraySync(void)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (g->host_only) return HDARRAY_OK;
    if (g->copy_stream) CUDA_TRY(cudaStreamSynchronize(g->copy_stream));
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return check_device_error();
}

int HDArrayGetLastError(void)
{
    if (!g) return HDARRAY_ERR_STATE;
    int e = g->last_error;
    g->last_error = 0;
    return e;
}

const char *HDArrayErrorString(int code)
{
    switch (code) {
    case HDARRAY_OK: return "ok";
    case HDARRAY_ERR_INVAL: return "invalid argument";
    case HDARRAY_ERR_NOMEM: return "out of memory";
    case HDARRAY_ERR_RACE: return "two devices define the same element in one call";
    case HDARRAY_ERR_RANGE: return "section outside the array";
    case HDARRAY_ERR_TIMEOUT: return "device-side wait timed out";
    case HDARRAY_ERR_CUDA: return "CUDA error";
    case HDARRAY_ERR_STATE: return "invalid state";
    case HDARRAY_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown error";
    }
}

static void to_user(const Box &b, int64_t *out)
{
    for (int d = 0; d < 3; d++) {
        out[d] = b.lo[d];
        out[3 + d] = b.hi[d];
    }
}

int HDArraySetRankMap(int ndev, const int32_t *rank_of_dev, int my_rank)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    if (!g->arrays.empty()) return HDARRAY_ERR_STATE;  // buffers are placed when arrays are used
    if (!rank_of_dev || ndev == 0) {
        g->rank_of_dev.clear();
        g->my_rank = 0;
        return HDARRAY_OK;
    }
    if (ndev != g->ndev || my_rank < 0) return HDARRAY_ERR_INVAL;
    for (int d = 0; d < ndev; d++)
        if (rank_of_dev[d] < 0) return HDARRAY_ERR_INVAL;
    g->rank_of_dev.assign(rank_of_dev, rank_of_dev + ndev);
    g->my_rank = my_rank;
    g->memo.clear();  // plans compiled for another placement
    return HDARRAY_OK;
}

int HDArraySetTransport(HDArrayTransport_t fn, void *user)
{
    if (!g || !g->inited) return HDARRAY_ERR_STATE;
    g->transport = fn;
    g->transport_user = user;
    return HDARRAY_OK;
}

int64_t HDArrayGetRankPlan(HDArray_t *hA, int64_t *out, int64_t cap)
{
    if (!g || !hA || !g->arrays.count(hA)) return HDARRAY_ERR_INVAL;
    std::vector<int64_t> recs;
    rank_records(hA, hA->last_moves, recs);
    const int64_t n = (int64_t)(recs.size() / HDARRAY_RANK_RECORD);
    if (out)
        for (int64_t i = 0; i < n && i < cap; i++)
            memcpy(out + HDARRAY_RANK_RECORD * i, recs.data() + HDARRAY_RANK_RECORD * i,
                   sizeof(int64_t) * HDARRAY_RANK_RECORD);
    return n;
}

// Boxes and 16-byte aligned staging offsets of transport records; the total bytes, or < 0.
static int64_t staging_layout(const HDArray *a, int64_t nrec, const int64_t *recs, std::vector<Box> &boxes,
                              std::vector<int64_t> &offs)
{
    if (nrec < 0 || (nrec > 0 && !recs)) return HDARRAY_ERR_INVAL;
    int64_t total = 0;
    for (int64_t i = 0; i < nrec; i++) {
        const int64_t *r = recs + HDARRAY_RANK_RECORD * i;
        if (r[0] < 0 || r[0] >= g->ndev || r[1] < 0 || r[1] >= g->ndev) return HDARRAY_ERR_INVAL;
        Box b;
        for (int d = 0; d < 3; d++) {
            b.lo[d] = r[4 + d];
            b.hi[d] = r[7 + d];
            const int64_t n = d < a->dim ? a->n[d] : 1;
            if (b.lo[d] < 0 || b.hi[d] > n || b.hi[d] <= b.lo[d]) return HDARRAY_ERR_RANGE;
        }
        total = (total + 15) / 16 * 16;
        offs.push_back(total);
        boxes.push_back(b);
        total += b.volume() * a->esize;
    }
    return total;
}

int64_t HDArrayStagingBytes(HDArray_t *hA, int64_t nrec, const int64_t *recs)
{
    if (!g || !hA || !g->arrays.count(hA)) return HDARRAY_ERR_INVAL;
    std::vector<Box> boxes;
    std::vector<int64_t> offs;
    return staging_layout(hA, nrec, recs, boxes, offs);
}

// Copy the records' boxes between the local devices' buffers and the staging buffer.
static int pack_unpack(HDArray *a, int64_t nrec, const int64_t *recs, char *staging, int64_t bytes, bool pack)
{
    if (!g || !g->inited || !a || !g->arrays.count(a)) return HDARRAY_ERR_INVAL;
    if (g->host_only) return HDARRAY_ERR_UNSUPPORTED;
    if (g->recording) return HDARRAY_ERR_STATE;
    std::vector<Box> boxes;
    std::vector<int64_t> offs;
    const int64_t total = staging_layout(a, nrec, recs, boxes, offs);
    if (total < 0) return (int)total;
    if (nrec == 0) return HDARRAY_OK;
    if (!staging || bytes < total) return HDARRAY_ERR_RANGE;
    int jrc = join_write(a);
    if (jrc) return jrc;
    std::vector<CopyTask> tasks;
    for (int64_t i = 0; i < nrec; i++) {
        const int dev = (int)recs[HDARRAY_RANK_RECORD * i + (pack ? 0 : 1)];
        if (!is_local(dev)) return HDARRAY_ERR_INVAL;
        const DevBuf &b = a->buf[dev];
        if (!b.ptr || !box_contains(b.alloc, boxes[i])) return HDARRAY_ERR_RANGE;
        DevBuf st;  // the record's stretch of staging, seen as a dense buffer over its box
        st.alloc = boxes[i];
        set_strides(a, st);
        st.ptr = staging + offs[i];
        if (pack) copy_tasks(a, b, st, boxes[i], tasks);
        else copy_tasks(a, st, b, boxes[i], tasks);
    }
    std::shared_ptr<DevMem> mem;
    std::vector<const char *> addr;
    int rc = upload({{tasks.data(), tasks.size() * sizeof(CopyTask)}}, mem, addr);
    if (rc) return rc;
    LaunchRec L;
    L.kind = L_COPY;
    L.p0 = addr[0];
    L.n0 = (int64_t)tasks.size();
    rc = issue_recorded(L);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(g->stream));  // the task table is freed on return
    return HDARRAY_OK;
}

int HDArrayPackBoxes(HDArray_t *hA, int64_t nrec, const int64_t *recs, void *staging, int64_t bytes)
{
    return pack_unpack(hA, nrec, recs, (char *)staging, bytes, true);
}

int HDArrayUnpackBoxes(HDArray_t *hA, int64_t nrec, const int64_t *recs, const void *staging, int64_t bytes)
{
    return pack_unpack(hA, nrec, recs, (char *)const_cast<void *>(staging), bytes, false);
}

int64_t HDArrayGetPlan(HDArray_t *hA, int64_t *out, int64_t cap)
{
    if (!g || !hA || !g->arrays.count(hA)) return HDARRAY_ERR_INVAL;
    const auto &mv = hA->last_moves;
    for (int64_t i = 0; i < (int64_t)mv.size() && i < cap && out; i++) {
        out[8 * i] = mv[i].src;
        out[8 * i + 1] = mv[i].dst;
        to_user(mv[i].box, out + 8 * i + 2);
    }
    return (int64_t)mv.size();
}

int64_t HDArrayGetGDEF(HDArray_t *hA, int p, int q, int64_t *out, int64_t cap)
{
    if (!g || !hA || !g->arrays.count(hA) || p < 0 || q < 0) return HDARRAY_ERR_INVAL;
    const GState &s = hA->states[hA->cur];
    if (p >= (int)s.own.size() || q >= (int)s.own.size() || p == q) return 0;
    BoxSet x = set_intersect(s.own[p], s.stale[q]);
    for (int64_t i = 0; i < (int64_t)x.size() && i < cap && out; i++) to_user(x[i], out + 6 * i);
    return (int64_t)x.size();
}

int HDArrayGetDeviceBuffer(HDArray_t *hA, int dev, void **ptr, int64_t *lo, int64_t *hi, int64_t *strides)
{
    if (!g || !hA || !g->arrays.count(hA) || dev < 0 || !ptr) return HDARRAY_ERR_INVAL;
    *ptr = nullptr;
    if (hA->write_pending) {  // the caller may read the memory at once
        if (cudaEventSynchronize(hA->write_ev) != cudaSuccess) {
            cudaGetLastError();
            return HDARRAY_ERR_CUDA;
        }
        hA->write_pending = false;
    }
    if (dev >= (int)hA->buf.size()) return HDARRAY_OK;
    const DevBuf &b = hA->buf[dev];
    *ptr = b.ptr;
    for (int d = 0; d < 3; d++) {
        if (lo) lo[d] = b.alloc.lo[d];
        if (hi) hi[d] = b.alloc.hi[d];
        if (strides) strides[d] = b.st[d];
    }
    return HDARRAY_OK;
}

int HDArrayReadDeviceBuffer(HDArray_t *hA, int dev, const int64_t *lo, const int64_t *hi, void *out)
{
    if (!g || !g->inited || !hA || !g->arrays.count(hA) || dev < 0 || !lo || !hi || !out)
        return HDARRAY_ERR_INVAL;
    if (g->host_only) return HDARRAY_ERR_STATE;
    if (dev >= (int)hA->buf.size() || !hA->buf[dev].ptr) return HDARRAY_ERR_RANGE;
    const DevBuf &b = hA->buf[dev];
    Box bx = make_box(0, 0, 0, 1, 1, 1);
    for (int d = 0; d < hA->dim; d++) {
        bx.lo[d] = lo[d];
        bx.hi[d] = hi[d];
    }
    if (bx.empty()) return HDARRAY_OK;
    if (!box_contains(b.alloc, bx)) return HDARRAY_ERR_RANGE;
    const int jrc = join_write(hA);
    if (jrc) return jrc;
    // view `out` as a dense array shaped like the box: a one-box "user array"
    HDArray tmp;
    tmp.dim = hA->dim;
    tmp.esize = hA->esize;
    for (int d = 0; d < 3; d++) tmp.n[d] = bx.hi[d] - bx.lo[d];
    DevBuf shifted = b;
    for (int d = 0; d < 3; d++) {
        shifted.alloc.lo[d] -= bx.lo[d];
        shifted.alloc.hi[d] -= bx.lo[d];
    }
    Box local = make_box(0, 0, 0, tmp.n[0], tmp.n[1], tmp.n[2]);
    int rc = memcpy_box(&tmp, shifted, local, out, false);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(g->stream));
    return HDARRAY_OK;
}

int HDArrayGetCounters(int64_t *out, int n)
{
    if (!g || !out || n < 0) return HDARRAY_ERR_INVAL;
    for (int i = 0; i < n && i < 5; i++) out[i] = g->counters[i];
    return HDARRAY_OK;
}

}  // extern "C"
