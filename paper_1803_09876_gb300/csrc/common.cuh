// Internal declarations shared by the library's translation units: status
// handling, the pluggable device allocator, handle layouts.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <memory>
#include <vector>

#include "../../include/jsweep.h"

namespace js {

// ---- status ------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

struct Status {
    int code = JSWEEP_OK;
    bool ok() const { return code == JSWEEP_OK; }
};

#define JS_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::js::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                            __FILE__, __LINE__);                                        \
            return e_ == cudaErrorMemoryAllocation ? JSWEEP_ERR_OOM : JSWEEP_ERR_CUDA;  \
        }                                                                               \
    } while (0)

#define JS_TRY(expr)              \
    do {                          \
        int rc_ = (expr);         \
        if (rc_ != JSWEEP_OK)     \
            return rc_;           \
    } while (0)

// Kernel launches made by this library (reported per call in jsweep_timing).
extern std::atomic<int64_t> g_kernel_launches;
inline void note_launches(int64_t n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// Check the launch just made and count it.
#define JS_LAUNCH_CHECK() \
    do {                  \
        ::js::note_launches(1); \
        JS_CUDA(cudaGetLastError()); \
    } while (0)

// ---- device memory ------------------------------------------------------------
void *dev_alloc(size_t bytes, cudaStream_t s);   // NULL on failure (error message set)
void dev_free(void *p, size_t bytes, cudaStream_t s);

// Owning device buffer routed through the library allocator.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    jsweep_free_fn free_fn = nullptr;  // allocator that produced p (nullptr = cudaFree)
    void *free_ctx = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    int alloc(size_t nbytes, cudaStream_t s);     // frees the old buffer first
    int ensure(size_t nbytes, cudaStream_t s);    // grow only
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---- handles ------------------------------------------------------------------
constexpr int kMaxFaces = 7;  // faces per cell; bit 7 of the incoming mask flags a lagged face

// Compact patches of a mesh (JSWEEP_MODE_PATCH), built once per target size.
struct PatchPart {
    int target = 0;
    int64_t NP = 0;
    int maxP = 0;                 // cells in the largest patch
    std::vector<int32_t> ptr;     // host copy of d_ptr
    DevBuf d_ptr;                 // int32 [NP+1]: patch p holds cells d_ids[ptr[p] .. ptr[p+1])
    DevBuf d_ids;                 // int32 [N]: cells by patch, ascending id inside a patch
    DevBuf d_pof;                 // int32 [N]: patch of a cell
    DevBuf d_loc;                 // int32 [N]: position of a cell inside its patch
    std::vector<int32_t> nbp;     // host [NP][kPatchNbrs]: neighbouring patches (-1 pads)
    std::vector<int32_t> okey;    // host [8][NP]: lowest octant-diagonal level of each patch (-1: none)
    DevBuf d_nbp;
};
constexpr int kPatchNbrs = 64;    // neighbours tracked per patch (dependency counters)

struct Mesh {
    std::atomic<int> refs{1};
    int64_t N = 0, F = 0, Fb = 0;
    int FS = 0;  // face slots per cell = max faces per cell
    int GS = 0;  // slots per cell in the geometry records (FS padded to 4 or 8)
    DevBuf sface;    // int32 [N][FS]: (face id << 1) | (cell is cell1), -1 = empty slot
    DevBuf nbr;      // int32 [N][FS]: neighbour id, -(b+1) for boundary face b, INT32_MIN empty
    DevBuf nbr8;     // int32 [N][8]: the same padded to 8 slots (two 16-byte loads per cell)
    DevBuf normal;   // double [F][3]
    DevBuf geo32;    // float4 [N][GS]: outward vector area (a n, oriented out of the cell), w = nbr bits
    DevBuf geo64;    // double4 [N][GS]: outward vector area, w = nbr as double bits
    DevBuf vol64;    // double [N]
    DevBuf vol32;    // float [N]
    std::unique_ptr<PatchPart> part;  // lazily built (patch programs)
};

struct Quad {
    std::atomic<int> refs{1};
    int64_t M = 0;
    std::vector<double> dirs, w;  // host copies
    DevBuf dirs64;  // double [M][3]
    DevBuf dirs32;  // float4 [M]
    DevBuf w64;     // double [M]
    DevBuf w32;     // float [M]
};

struct UnitTable {
    int mode = -1, priority = -1, cluster = -1, stagger = -1, order = -1;
    int64_t warps = 0;             // patch tasks: the launch's warp count (unit t runs on warp t mod warps)
    DevBuf units;                  // int4 [n_units]: (m, pos0, ncells, wait target)
    int64_t n_units = 0;
    std::vector<int64_t> slot_ptr; // level-sync: units of level l are [slot_ptr[l], slot_ptr[l+1])
    bool dirmajor = false;         // persistent queues: units direction by direction, each in layer order
    DevBuf dir_ptr;                // int64 [M+1]: units of direction m are [dir_ptr[m], dir_ptr[m+1])
};

// Patch-program schedule of a handle (JSWEEP_MODE_PATCH).
struct PatchSched {
    int target = 0;
    int64_t NP = 0, n_tasks = 0, cap = 0;
    int n_oct_max = 0;            // most directions in one octant
    DevBuf entries;               // uint16 [M][N]: per direction, cells by (patch, level, id):
                                  //   position inside the patch | bit 15 = first cell of a new level
    DevBuf pmask;                 // uint8 [M][N]: incoming-face mask of each entry
    DevBuf seg;                   // int32 [M][NP+1]: entries of (direction, patch)
    DevBuf oct_dirs;              // int32 [8][n_oct_max]: directions of each octant
    DevBuf oct_n;                 // int32 [8]
    DevBuf q_init;                // int32 [n_tasks]: tasks (octant * NP + patch) in dispatch order
    DevBuf queue;                 // int32 [cap]
    DevBuf seq;                   // uint32 [cap]: slot i holds a task once seq = i + 1
    DevBuf ctr;                   // uint32 [4]: dispatched, queued, finished, re-queued
    DevBuf prog;                  // int32 [8 * NP][n_oct_max]: entries done per (task, direction)
    DevBuf cnt_init, cnt;         // int32 [8 * NP]: upstream programs still to finish
    DevBuf down_ptr, down;        // CSR [8 * NP + 1] / [edges]: downstream programs
    int64_t n_ready0 = 0;         // programs queued at the start (no upstream program)
    int64_t last_requeued = 0;
};

struct Dags {
    std::atomic<int> refs{1};  // the handle and every batch problem that uses it
    int eager_cap = 0;         // cells an eager (not stalled) cycle search may visit; 0 = cycle_search_max
    Mesh *mesh = nullptr;
    Quad *quad = nullptr;
    jsweep_options opt{};
    int64_t N = 0, M = 0, Lmax = 0, T = 0;  // T = lagged (face, dir) pairs
    std::vector<int64_t> nlevels;  // [M]
    std::vector<int64_t> lp_off;   // [M+1] offsets of each direction's level_ptr in lp
    std::vector<int64_t> lag_ptr_h;  // [M+1]
    DevBuf level;   // int32 [M][N] (cell order)
    DevBuf order;   // int32 [M][N]
    DevBuf mask;    // uint8 [M][N] (level order): incoming-face bits, bit 7 = a lagged face
    DevBuf lp;      // int32 [sum (L_m + 1)]
    DevBuf lag_ptr; // int32 [M+1]
    DevBuf lag_m, lag_face, lag_up, lag_dn;  // int32 [T], sorted by (m, face)
    // schedule layering used by the sweeps (levels, or octant-aligned layers)
    int layering = JSWEEP_LAYERS_LEVEL;
    int64_t Smax = 0;                 // largest layer count
    std::vector<int64_t> slayers;     // [M] layer count per direction
    std::vector<int64_t> sp_off;      // [M+1] offsets into the layer pointers
    DevBuf korder, kmask, klp;        // octant layering: order, mask, layer pointers
    const int32_t *s_order = nullptr; // the order / mask / layer pointers in use
    const uint8_t *s_mask = nullptr;
    const int32_t *s_lp = nullptr;
    // lagged upwind values: [T][R] in the precision of the last sweep
    DevBuf psi_lag;
    int lag_R = 0, lag_prec = -1;
    // sweep workspaces
    DevBuf psi;      // [N][M][R] (cell-major: a cell's directions are contiguous)
    DevBuf srcv;     // [N][RS] source records: S V for each rhs, then sigma_t V (see src_stride)
    DevBuf inflow;   // [R][Fb] copy (stable pointer for graphs)
    DevBuf phi_a, phi_b;  // [R][N] (SI ping-pong)
    DevBuf red;      // residual accumulators / flags
    DevBuf counters; // persistent schedule: error word
    DevBuf qstate;   // persistent queues: per-direction cursor and finished-unit counter
    DevBuf flags;    // int32 [N][M]: sweep epoch at which (cell, direction) was last written
    int epoch = 0;
    DevBuf dirs4_64; // double [M][4]: directions padded for aligned loads (FP64 sweeps)
    // face-coefficient streams of the level-synchronous sweeps, [0] FP32 and [1]
    // FP64 (see coef_record_bytes); each lives as long as the handle, so batch
    // problems may keep its address
    struct FaceStream {
        DevBuf buf;
        int maxf = 0;
        const int32_t *order = nullptr;  // the order and directions it was built for
        const void *dirs = nullptr;
        bool failed = false;             // allocation refused: sweeps read the cell geometry
    } coef[2], pcoef[2];                 // pcoef: interior neighbours as positions in the sweep order
    // psi in each direction's sweep order ([M][N][R], level-synchronous sweeps with
    // pcoef); prec/R of its contents, failed when its allocation was refused
    DevBuf psi_seq;
    bool psi_seq_failed = false;
    // tail of the level-synchronous sweep (the last, small slots: one block per direction)
    DevBuf tail_lpoff;       // int64 [M+1]: device copy of sp_off
    DevBuf tail_nlev;        // int32 [M]: device copy of slayers
    UnitTable ut;
    std::unique_ptr<PatchSched> ps;  // lazily built (patch programs)
    // CUDA graph of the level-synchronous sweep
    cudaGraphExec_t graph = nullptr;
    std::string graph_key;
    cudaStream_t capture_stream = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    jsweep_timing timing{};
    ~Dags();
};

void mesh_release(Mesh *m);
void quad_release(Quad *q);
void dags_release(Dags *d);

// dag build (dag_build.cu)
int build_dags(Dags *d, cudaStream_t s);
// Graphs of the eight octant diagonals (1/sqrt3)(+-1, +-1, +-1) of d's mesh
// (levels only; direction o has the sign bits of octant o); nullptr on failure.
Dags *build_diagonals(Dags *d, cudaStream_t s);

// unit schedules and sweeps (sweep.cu)
// dirmajor: the persistent queues' direction-major table (single problems);
// otherwise the slot-ordered table (level-synchronous sweeps, batches, patch tasks)
int ensure_units(Dags *d, int mode, int max_cells, cudaStream_t s, int64_t resident_warps = 0,
                 bool dirmajor = false);
int ensure_dirs64x4(Dags *d, DevBuf &buf, cudaStream_t s);  // FP64 directions as [M][4]
// Face-coefficient stream of a handle (level-synchronous sweeps), built on
// first use; nullptr when the option is off or its allocation was refused.
const unsigned char *ensure_face_stream(Dags *d, int prec, cudaStream_t s, bool positions = false);
int run_sweep(Dags *d, int nrhs, int prec, const void *sigma_t, const void *ang_source,
              const void *inflow, void *phi_out, void *psi_out, cudaStream_t s);
int run_source_iteration(Dags *d, int nrhs, int prec, const void *sigma_t, const void *c_ratio,
                         const void *q, const void *inflow, double tol, int max_iters,
                         void *phi_out, int *iters_out, double *resid_out, cudaStream_t s);
int run_source_iteration_mg(Dags *d, int n_groups, int prec, const void *sigma_t, const void *sigma_s,
                            const void *q, const void *inflow, double tol, int max_iters, void *phi_out,
                            int *iters_out, double *resid_out, cudaStream_t s);

// shared device helpers
int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
int radix_sort_segments(const uint32_t *keys_in, int64_t n_seg, int64_t seg_len, int key_bits,
                        const int32_t *vals_in, int32_t *vals_out, uint32_t *keys_out,
                        cudaStream_t s);

inline int grid_for(int64_t n, int block, int64_t cap = 1 << 20) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int device_sm_count();
int device_clock_khz();  // SM clock of the current device (cached)
unsigned long long *bounds_word();  // error word of the bounds-checked build (nullptr otherwise)
int check_options(const jsweep_options *opt, jsweep_options *o);

}  // namespace js

// The opaque handles of the C ABI point at these objects.
inline js::Mesh *impl(jsweep_mesh_t h) { return reinterpret_cast<js::Mesh *>(h); }
inline js::Quad *impl(jsweep_quad_t h) { return reinterpret_cast<js::Quad *>(h); }
inline js::Dags *impl(jsweep_dags_t h) { return reinterpret_cast<js::Dags *>(h); }
