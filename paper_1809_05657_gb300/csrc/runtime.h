// runtime.h -- internal structures of the HDArray runtime (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

#include "hdarray.h"
#include "kernels.h"
#include "sections.h"

struct HDArray;

namespace hda {

struct Offset {
    int32_t o[3];
};

enum KKind { K_JACOBI2D, K_COPY, K_STENCIL3D, K_SQDIFF, K_GEMM, K_TRMM, K_EXCHANGE, K_CONV2D, K_COLMEAN, K_CENTER, K_SYRK, K_SYMM, K_COLNORM, K_COLSCALE, K_USER };

// A built-in kernel: its arguments and the use/def offsets of each array argument, the table the
// paper's frontend builds from the pragma clauses (Sec. 4.1).
struct KernelDef {
    std::string name;
    KKind kind;
    int narr = 0;
    int nscal_f = 0;  // floating scalars (read as double from varargs)
    int nscal_i = 0;  // integer scalars (read as int from varargs)
    int space = 0;    // the argument whose index space the work partition covers
    std::vector<std::vector<Offset>> use, def;  // per array argument
    uint64_t version = 1;
    HDArrayLauncher_t launcher = nullptr;  // user kernels (HDArrayRegisterKernel)
    void *user = nullptr;
};

// A device buffer: the box of coordinates it covers and element strides of dimensions 0..2.
struct DevBuf {
    char *ptr = nullptr;
    Box alloc = {};
    int64_t st[3] = {0, 0, 0};
    size_t bytes = 0;
};

// GDEF bookkeeping of one array in factored form: own[p] = elements whose last writer is device
// p; stale[p] = elements device p does not hold.  sGDEF_{p,q} = own[p] n stale[q] and
// rGDEF_{q,p} = sGDEF_{p,q}.
struct GState {
    std::vector<BoxSet> own, stale;
    uint64_t hash = 0;
};

struct Move {
    int src, dst;
    Box box;
};

struct Part {
    int dim = 0;
    int64_t n[3] = {1, 1, 1};
    int nparts = 0;
    std::vector<Box> box;  // per device (may be empty)
};

// One kernel launch, recorded so that batches can merge it and graphs can replay it.
enum LKind { L_COPY, L_JACOBI2D, L_SQDIFF, L_GEMM64, L_STENCIL3D, L_GEMM_TC, L_SPLIT, L_GEMM_PANEL, L_FLAT2D, L_FLAT3D, L_CONV2D,
             L_COLMEAN, L_CENTER, L_SYMM, L_USER };
struct LaunchRec {
    int kind = 0;
    int dtype = 0;
    const void *p0 = nullptr, *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;
    const void *p4 = nullptr;      // a convolution's weights when p3 holds the tensor maps
    const void *p1_alt = nullptr;  // the same tiles in the reverse order (alternating launches)
    bool alt_calls = false;        // successive calls of the plan alternate p1 and p1_alt
    int64_t n0 = 0, n1 = 0, n2 = 0, n3 = 0;
    double f0 = 0, f1 = 0;
};
cudaError_t issue(const LaunchRec &L, cudaStream_t s);

// Device memory owned by a plan (the packed descriptor tables its launches read).
struct DevMem {
    void *ptr = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    ~DevMem();
};

// Host copies of a fused stencil plan's tables, kept so that a batch can concatenate them.
struct Sten2DHost {
    int dtype = 0;
    int variant = 1;    // kernel variant of the tiles (0, 1 warp tiles; 2 flat; 3 packed streams;
                        // 5 rows staged by bulk tensor copies)
    int warps = 8;      // warps per CTA of the warp variants
    bool flat = false;  // flat-block tiles (k_jacobi2d_flat)
    size_t smem = 0;    // dynamic shared memory per CTA (flat, packed-stream and TMA forms)
    std::vector<StenPart2D> parts;
    std::vector<StenTile2D> tiles;
    std::vector<Seg> segs;
    std::vector<CUtensorMap> maps;  // TMA variant: one per part (its X buffer)
    bool map_error = false;
    int rx_cap = 0;  // TMA variant: received elements a tile keeps to patch its first stages (0: none)
};
struct Sten3DHost {
    int dtype = 0;
    bool flat = false;
    size_t smem = 0;
    std::vector<StenPart3D> parts;
    std::vector<StenTile3D> tiles;
    std::vector<Seg> segs;
    std::vector<CUtensorMap> maps;  // TMA variant: one per part (its X buffer)
    bool map_error = false;
};

struct ArrStep {
    HDArray *a = nullptr;
    int pre = 0, post = 0;
    std::vector<Move> moves;
    bool used = false, defined = false;
};

// A cached call: the communication of one HDArrayApplyKernel signature from one GDEF state
// (Sec. 4.2: the intersections are cached per kernel call and partition and reused while LUSE and
// GDEF are unchanged), plus the compiled launches.
struct Plan {
    uint64_t id = 0;
    const KernelDef *k = nullptr;
    int part = 0;
    std::vector<HDArray *> args;
    std::vector<double> scal;
    std::vector<std::vector<BoxSet>> luse, ldef;  // per argument, per device
    std::vector<ArrStep> steps;                   // per distinct array
    // compiled form
    std::string compiled_sig;
    std::vector<LaunchRec> launches;
    std::shared_ptr<DevMem> tables;
    bool fused = false;
    std::vector<CopyTask> copy_host;  // exchange tasks (batch merging)
    Sten2DHost s2;                    // stencil tables (batch merging)
    Sten3DHost s3;
    std::shared_ptr<DevMem> panels;   // pre-split bf16 operand panels (tensor-core GEMM)
    std::shared_ptr<DevMem> extra_tables;  // descriptor tables of the panel launches
    uint64_t split_version[2] = {~0ull, ~0ull};  // content versions of A and B the panels hold
    std::vector<HDArrayWork_t> user_work;         // a user kernel's per-device work
    bool alt = false;                             // next call takes the launches' p1_alt tables
    std::shared_ptr<DevMem> red;  // residual plans: per-CTA partials, counter and the sum of R
};

// Layout of a residual plan's `red` scratch for nblocks CTAs: partials, then the counter, then the
// sum of the values the launch stored.
inline size_t red_counter_offset(int64_t nblocks) { return (size_t)((nblocks * 8 + 255) / 256 * 256); }
inline size_t red_bytes(int64_t nblocks) { return red_counter_offset(nblocks) + 256; }

// Device memory: cudaMalloc / cudaFree, or the allocator set with HDArraySetAllocator (each
// allocation is released by the allocator that provided it).
int dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
int set_allocator(HDArrayAlloc_t alloc, HDArrayFree_t free_fn, void *user);
int user_launch_rc();  // the failure code of the last user launcher that failed

}  // namespace hda

struct HDArray {
    std::string sym;
    int dtype = 0;
    int esize = 0;
    int dim = 0;
    int64_t n[3] = {1, 1, 1};
    int P = 0;
    std::vector<hda::DevBuf> buf;
    std::vector<hda::GState> states;
    int cur = 0;
    uint64_t generation = 1;  // bumps when the state table is reset
    uint64_t epoch = 1;       // bumps when any device buffer moves
    uint64_t version = 0;     // bumps whenever any element is (re)defined
    uint64_t uid = 0;
    std::vector<hda::Move> last_moves;
    // asynchronous Write from host memory (on the library's copy stream): write_ev marks its end,
    // which library work on the array waits for; use_ev marks the end of the library stream's last
    // work on the array, which the next asynchronous Write waits for (recorded once track_use is set)
    cudaEvent_t write_ev = nullptr, use_ev = nullptr;
    bool write_pending = false, track_use = false;
};
