#include <cstdlib>
// Per-direction dependency-graph build on the device (Sec. V-A; Listing 1
// init/input/compute readiness), with cycle breaking and the level-major
// reorder.
//
// Data layout: the frontier and candidate lists are per direction ([M][N]).
// The per-(direction, cell) state of the frontier loop (masks, state words
// holding the count and the level, stamps, claims) is [S / 8][N][8] over
// direction slots: the directions of an
// octant get consecutive slots (each octant padded to a multiple of 8), so one
// 32-byte sector holds a cell's state in 8 directions of one octant.  Those
// directions peel nearly the same cells at nearly the same step, so their
// scattered accesses share sectors in L2 instead of each missing to DRAM.  The
// levels and masks are transposed to [M][N] after the loop.
//
// Steps:
//   1. classify  (one thread per (m, c)): upwind/downwind role of each face of
//      c from the FP64 sign of ((n_x O_x) + (n_y O_y)) + (n_z O_z) with
//      round-to-nearest multiplies and adds (no FMA contraction), so that the
//      signs are bit-identical to any IEEE evaluation in that order.  Yields
//      the incoming-face mask, the outgoing active-edge mask and the count of
//      unfinished upwind cells (Listing 1, init).
//   2. peel      (frontier per direction): a ready cell gets
//      level = 1 + max(level of its active upwind cells) and decrements its
//      downwind cells' counts; a count reaching zero makes that cell ready
//      (Listing 1, compute/input).  Levels are longest-path levels.
//   3. resolve   (only for a direction whose frontier ran empty while cells
//      remain, i.e. the rest is blocked by cycles): from cells that were
//      touched since the last stall, follow "first unfinished upwind cell"
//      pointers until they close a loop; that loop lies in a strongly
//      connected component S.  The set of unfinished cells that reach the loop
//      backwards is gathered under a size cap; when it closes, S is computed
//      exactly inside it and the active face of smallest id inside S is
//      lagged.  Lags found in one step are applied after the step, so every
//      search sees the same graph.  Any order of lagging components gives the
//      same final lag set as "lag the smallest face in every component, then
//      recompute components, until acyclic": the components of the graph after
//      a lag refine the components before it, and each component's own
//      recursion depends only on the edges inside it.
//   4. sort      cells of each direction by (level, cell id) with a stable
//      LSD radix sort; level_ptr from the sorted keys; the incoming mask is
//      gathered into level order (bit 7 flags a cell with a lagged face).
#include <climits>
#include <cstring>
#include <memory>

#include "common.cuh"

namespace js {

namespace {

constexpr int kWarp = 32;

__device__ __forceinline__ double dot_rn(const double *n, const double *o) {
    double a = __dmul_rn(n[0], o[0]);
    double b = __dmul_rn(n[1], o[1]);
    double c = __dmul_rn(n[2], o[2]);
    return __dadd_rn(__dadd_rn(a, b), c);
}

// Sign of dot_rn(n, o).  Out of line: called only where the FP32 evaluation
// cannot decide the sign, so the (slow) FP64 arithmetic is not issued for
// every face and direction.
__device__ __noinline__ int sign_dot_rn(const double *n, const double *o) {
    const double d = dot_rn(n, o);
    return d > 0.0 ? 1 : (d < 0.0 ? -1 : 0);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

struct BuildCtx {
    int64_t N, M;
    int FS;
    const int32_t *sface, *nbr;
    const int4 *nbr8;  // [N][2]: neighbour ids padded to 8 slots
    const double *normal, *dirs;
    int32_t *st;  // state words (st_count, st_level)
    int32_t *stamp, *claim;
    uchar4 *msk;  // [M][N]: x = incoming-face bits, y = outgoing active-edge bits, z = lagged-face bits
                  // (one 4-byte record, so a cell's three masks cost one scattered access)
    int32_t *front;   // [2][M][N]
    int32_t *nfront;  // [2][M]
    int32_t *cand;    // [2][M][N]
    int32_t *ncand;   // [2][M]
    int32_t *cidx, *epoch, *nproc;  // [M]
    int4 *pend;
    int32_t *npend;
    int64_t pend_cap;
    int4 *lagall;
    int32_t *nlag;
    int64_t lag_cap;
    int32_t *status;  // [0] error code, [1] error info, [2] remaining (clamped), [3] step counter,
                      // [4] stall rounds, [5] cycles found by walks, [6] components lagged
    int32_t *ticket;  // blocks of the running peel that have read its frontier counts
    unsigned long long *wclaim;  // [M][N]: (epoch << 32) | (walker + 1) of the walk that owns the cell
    // acyclicity certificate: a direction in which the level of its octant's
    // diagonal (lam) increases along every edge has no cycle, so it needs no
    // cycle candidates or resolution.  cyc[m] = 1 when not certified.
    int32_t *seeds;      // [M][kSeedCapG]: cells at which walks closed a pointer cycle this step
    int32_t *nseeds;     // [M]
    const int32_t *lam;  // [8][N] or null (no certificate: every direction is treated as cyclic)
    const int32_t *oct;  // [M]
    int32_t *cyc;        // [M]
    const int32_t *dslot;  // [M]: the direction's state slot (see the data layout above)
    const int32_t *sdir;   // [S]: direction of a slot, or -1 (padding)
    int64_t S;             // state slots (a multiple of 8)
};

// State word of a (direction, cell) in the frontier loop: bits 0-3 hold the
// number of its active upwind faces not yet processed, bits 4-31 its level,
// all ones (a negative word) until the cell is processed.  The count and the
// level of a cell then share one sector with the other directions of its
// group: the decrements by its upwind cells, its own level store and the
// level reads by its downwind cells all touch that one sector.  Levels fit
// while below 2^27; a longest path that long passes through the levels 2^24
// and above, which the build rejects after the loop ("too many levels").
constexpr int32_t kStUnset = (int32_t)0xFFFFFFF0u;
__device__ __forceinline__ int32_t st_count(int32_t w) { return w & 15; }
__device__ __forceinline__ int32_t st_level(int32_t w) { return w < 0 ? -1 : w >> 4; }

// Index of direction m's state of cell v: [slot / 8][N][8].
struct StateIx {
    int64_t b;
    __device__ __forceinline__ int64_t operator()(int32_t v) const { return b + 8 * (int64_t)v; }
};
__device__ __forceinline__ StateIx state_ix(const BuildCtx &c, int64_t m) {
    const int s = c.dslot[m];
    return StateIx{(int64_t)(s >> 3) * c.N * 8 + (s & 7)};
}

__device__ __forceinline__ void push(int32_t *list, int32_t *count, int32_t v, int64_t cap,
                                     int32_t *status) {
    int32_t i = atomicAdd(count, 1);
    if (i < cap) {
        list[i] = v;
    } else {
        atomicCAS(&status[0], 0, JSWEEP_ERR_OOM);
    }
}

// Slots for na items in list A (counter ca) and nb items in list B (counter
// cb) for every active lane; lanes with the same key use the same counters and
// must be contiguous, and the active lanes must be a prefix of the warp.  One
// atomic per counter and key, both in flight together.  Returns each lane's
// first slot in ra / rb.
__device__ __forceinline__ void warp_reserve2(int32_t *ca, int32_t *cb, int na, int nb, uint64_t key, int32_t &ra,
                                              int32_t &rb) {
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    int xa = na, xb = nb;  // inclusive scans over the active lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ya = __shfl_up_sync(act, xa, o), yb = __shfl_up_sync(act, xb, o);
        if (lane >= o) {
            xa += ya;
            xb += yb;
        }
    }
    const unsigned peers = __match_any_sync(act, key);
    const int first = __ffs(peers) - 1, last = 31 - __clz(peers);
    const int a0 = __shfl_sync(act, xa - na, first), b0 = __shfl_sync(act, xb - nb, first);
    const int a1 = __shfl_sync(act, xa, last), b1 = __shfl_sync(act, xb, last);
    int32_t ba = 0, bb = 0;
    if (lane == first) {
        if (a1 > a0) ba = atomicAdd(ca, a1 - a0);
        if (b1 > b0) bb = atomicAdd(cb, b1 - b0);
    }
    ra = __shfl_sync(act, ba, first) + (xa - na - a0);
    rb = __shfl_sync(act, bb, first) + (xb - nb - b0);
}

// The first F neighbour slots of cell v (F <= 8; kernels are compiled for the
// mesh's face slots rounded up to 4, 6 or 7).
template <int F>
__device__ __forceinline__ void load_nbr(const BuildCtx &c, int32_t v, int32_t (&nb)[F]) {
    static_assert(F >= 4 && F <= 8, "face slots");
    const int4 a = __ldg(c.nbr8 + 2 * (int64_t)v);
    nb[0] = a.x; nb[1] = a.y; nb[2] = a.z; nb[3] = a.w;
    if constexpr (F > 4) {
        const int4 b = __ldg(c.nbr8 + 2 * (int64_t)v + 1);
        const int32_t bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 4; j < F; ++j) nb[j] = bb[j - 4];
    }
}

// Face classification, cell by cell (one thread per cell v, a loop over the
// directions in their state-slot groups of 8).  The cell's faces, neighbours
// and normals are read once for all directions.
// Sign of the FP64 expression ((n_x O_x) + (n_y O_y)) + (n_z O_z): the FP32
// evaluation of the same expression on the rounded inputs differs from the
// exact dot product by at most about 6 * 2^-24 * sum |n_i O_i| <= 4e-7 for unit
// vectors, so when its magnitude exceeds 1e-6 its sign is the exact sign, and
// so the sign of the FP64 evaluation (whose error is below 1e-15); otherwise the
// FP64 expression itself decides.  The signs are those of the FP64 evaluation
// in every case.
// List pushes: the pushes of a warp for a direction reserve their slots with
// one atomic (list order carries no meaning: levels are maxima over
// upwind cells and the lag rule picks the smallest face of a component,
// whatever order cells were found in).
constexpr int kClassifyThreads = 256;  // compiled for 3 blocks per SM (no spills): 9.4 -> 7.9 ms at 128^3

__global__ void __launch_bounds__(kClassifyThreads, 3) k_classify(BuildCtx c, const float *dirs32) {
    extern __shared__ unsigned char cls_smem[];
    uint8_t *sh_cyc = cls_smem;  // [M]: a back edge of the certificate seen in this block
    const int lane = threadIdx.x & 31;
    for (int64_t m = threadIdx.x; m < c.M; m += blockDim.x) sh_cyc[m] = 0;
    const int64_t v64 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = v64 < c.N;
    const int32_t v = live ? (int32_t)v64 : 0;
    // the cell's faces: FP32 normals oriented out of v, neighbours, face slots
    // (a cell's face slots are filled from slot 0 on; empty slots hold -1)
    float nx[kMaxFaces], ny[kMaxFaces], nz[kMaxFaces];
    int32_t nb[kMaxFaces], sf[kMaxFaces];
#pragma unroll
    for (int k = 0; k < kMaxFaces; ++k) {
        const int32_t q = (live && k < c.FS) ? c.sface[(int64_t)v * c.FS + k] : -1;
        sf[k] = q;
        nb[k] = q >= 0 ? c.nbr[(int64_t)v * c.FS + k] : -1;
        const double *n = c.normal + 3 * (int64_t)(q >= 0 ? q >> 1 : 0);
        nx[k] = q >= 0 ? (float)n[0] : 0.f;
        ny[k] = q >= 0 ? (float)n[1] : 0.f;
        nz[k] = q >= 0 ? (float)n[2] : 0.f;
    }
    // certificate back edges: bit 8 o + k when lam_o(v) <= lam_o(neighbour k)
    unsigned long long back = 0;
    if (c.lam && live) {
        for (int o = 0; o < 8; ++o) {
            const int32_t lv = c.lam[(int64_t)o * c.N + v];
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k)
                if (sf[k] >= 0 && nb[k] >= 0 && lv <= c.lam[(int64_t)o * c.N + nb[k]]) back |= 1ull << (8 * o + k);
        }
    }
    __syncthreads();
    // slot groups of 8 directions (block b starts at group b mod G, so that the
    // blocks' list counters are spread over the directions); the cell's masks
    // and state words of a group are stored as two full 32-byte sectors each
    const int64_t G = c.S / 8;
    const int64_t g0 = blockIdx.x % G;
    for (int64_t gi = 0; gi < G; ++gi) {
        const int64_t grp = g0 + gi < G ? g0 + gi : g0 + gi - G;
        if (live) {
            // the frontier loop's other state starts here too (whole sectors):
            // stamps, component claims and walk claims
            const int64_t w0 = (grp * c.N + v) * 8;
            uint4 *ps = reinterpret_cast<uint4 *>(c.stamp + w0);
            uint4 *pcl = reinterpret_cast<uint4 *>(c.claim + w0);
            uint4 *pw = reinterpret_cast<uint4 *>(c.wclaim + w0);
            const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
            ps[0] = zero;
            ps[1] = zero;
            pcl[0] = zero;
            pcl[1] = zero;
#pragma unroll
            for (int q = 0; q < 4; ++q) pw[q] = zero;
        }
        uint32_t wm[8], wc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            wm[j] = 0;
            wc[j] = 0;
            const int64_t m = c.sdir[grp * 8 + j];
            if (m < 0) continue;  // padding slot (uniform over the block)
            const float ox = __ldg(dirs32 + 3 * m), oy = __ldg(dirs32 + 3 * m + 1), oz = __ldg(dirs32 + 3 * m + 2);
            // signs of the FP64 expression, outward from each face's cell0: the
            // FP32 evaluation decides unless |d32| <= 1e-6 (bits of unc)
            int sgk[kMaxFaces];
            unsigned unc = 0;
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k) {
                const float d32 =
                    __fadd_rn(__fadd_rn(__fmul_rn(nx[k], ox), __fmul_rn(ny[k], oy)), __fmul_rn(nz[k], oz));
                sgk[k] = d32 > 0.f ? 1 : -1;
                if (sf[k] >= 0 && !(fabsf(d32) > 1e-6f)) unc |= 1u << k;
            }
            if (unc) {
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k)
                    if ((unc >> k) & 1u) sgk[k] = sign_dot_rn(c.normal + 3 * (int64_t)(sf[k] >> 1), c.dirs + 3 * m);
            }
            unsigned in = 0, out = 0;
            int count = 0;
            bool bin = false;
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k) {
                if (sf[k] < 0) continue;
                int sg = sgk[k];
                if (sf[k] & 1) sg = -sg;  // outward from v
                if (sg < 0) {
                    in |= 1u << k;
                    if (nb[k] >= 0) ++count;
                    else bin = true;
                } else if (sg > 0 && nb[k] >= 0) {
                    out |= 1u << k;
                }
            }
            wm[j] = in | (out << 8);  // uchar4 (in, out, 0, 0)
            wc[j] = (uint32_t)count;
            if (live) {
                // stamp (after the zeros above, same thread): epoch 1 is the first stall's candidate list
                if (count != 0 && bin) c.stamp[(grp * c.N + v) * 8 + j] = 1;
                const unsigned interior_in = in & (unsigned)(back >> (8 * (c.lam ? c.oct[m] : 0))) & 0xffu;
                if (interior_in) sh_cyc[m] = 1;  // an active edge against the diagonal's levels
            }
            // slots for the frontier (sources) and candidate lists: one atomic
            // per warp and list, only in the few warps that push
            const bool pf = live && count == 0, pc = live && count != 0 && bin;
            const unsigned bf = __ballot_sync(0xffffffffu, pf), bc = __ballot_sync(0xffffffffu, pc);
            if (bf | bc) {
                int gf = 0, gc = 0;
                if (lane == 0) {
                    if (bf) gf = atomicAdd(c.nfront + m, __popc(bf));
                    if (bc) gc = atomicAdd(c.ncand + m, __popc(bc));
                }
                gf = __shfl_sync(0xffffffffu, gf, 0);
                gc = __shfl_sync(0xffffffffu, gc, 0);
                if (pf || pc) {
                    const int off = pf ? gf + __popc(bf & lanemask_lt()) : gc + __popc(bc & lanemask_lt());
                    int32_t *list = (pf ? c.front : c.cand) + m * c.N;
                    if (off < c.N) list[off] = v;
                    else atomicCAS(&c.status[0], 0, JSWEEP_ERR_OOM);
                }
            }
        }
        if (live) {
            const int64_t w0 = (grp * c.N + v) * 8;
            uint4 *pm = reinterpret_cast<uint4 *>(reinterpret_cast<uint32_t *>(c.msk) + w0);
            uint4 *pc4 = reinterpret_cast<uint4 *>(c.st + w0);  // level unset, count
            const uint32_t u = (uint32_t)kStUnset;
            pm[0] = make_uint4(wm[0], wm[1], wm[2], wm[3]);
            pm[1] = make_uint4(wm[4], wm[5], wm[6], wm[7]);
            pc4[0] = make_uint4(u | wc[0], u | wc[1], u | wc[2], u | wc[3]);
            pc4[1] = make_uint4(u | wc[4], u | wc[5], u | wc[6], u | wc[7]);
        }
    }
    __syncthreads();
    for (int64_t m = threadIdx.x; m < c.M; m += blockDim.x)
        if (sh_cyc[m]) c.cyc[m] = 1;
}

// Exclusive offsets off[0..M] (shared memory) of per-direction counts
// count(m), computed by every block from the same counts, so that a step's
// work over all directions is spread evenly over a fixed grid.
template <class Count>
__device__ void block_offsets(int64_t M, Count count, int64_t *off) {
    __shared__ int64_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t per = (M + blockDim.x - 1) / blockDim.x;
    const int64_t lo = (int64_t)threadIdx.x * per, hi = min(lo + per, M);
    int64_t sum = 0;
    for (int64_t m = lo; m < hi; ++m) sum += count(m);
    int64_t x = sum;  // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int64_t run = x - sum + (warp ? wsum[warp - 1] : 0);
    for (int64_t m = lo; m < hi; ++m) {
        off[m] = run;
        run += count(m);
    }
    if (threadIdx.x == blockDim.x - 1) off[M] = run;
    __syncthreads();
}

// Direction of flat work index i: the largest m with off[m] <= i (off[M] > i).
__device__ __forceinline__ int64_t offset_owner(const int64_t *off, int64_t M, int64_t i) {
    int64_t lo = 0, hi = M;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One frontier step for every direction: the frontier cells of all
// directions, concatenated in direction order, are spread over the grid
// (dynamic shared memory: M + 1 offsets).  Block 0 also counts the step's
// cells into nproc (every frontier cell is processed exactly once), and the
// last block to have read the frontier counts clears them (the list they
// count is consumed) and stores the number of cells still to be processed.
template <int F>
__global__ void __launch_bounds__(256, 5) k_peel(BuildCtx c, int cur) {
    extern __shared__ int64_t peel_off[];
    const int nxt = cur ^ 1;
    const int32_t *nf = c.nfront + cur * c.M;
    const int64_t N = c.N;
    block_offsets(c.M, [&](int64_t m) { return (int64_t)min(nf[m], (int32_t)N); }, peel_off);
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *c.npend = 0;  // read by the last lag commit
        for (int64_t m = threadIdx.x; m < c.M; m += blockDim.x) c.nproc[m] += min(nf[m], (int32_t)N);
        __threadfence();  // the counts before block 0's ticket
    }
    const int64_t total = peel_off[c.M];
    {
        __shared__ int last;
        __shared__ long long rem_w[8];
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(c.ticket, 1) == (int)gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            __threadfence();
            long long rem = 0;
            for (int64_t m = threadIdx.x; m < c.M; m += blockDim.x) {
                rem += N - __ldcg(c.nproc + m);
                c.nfront[cur * c.M + m] = 0;
            }
            for (int o = 16; o > 0; o >>= 1) rem += __shfl_down_sync(0xffffffffu, rem, o);
            if ((threadIdx.x & 31) == 0) rem_w[threadIdx.x >> 5] = rem;
            __syncthreads();
            if (threadIdx.x == 0) {
                long long t = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += rem_w[w];
                c.status[2] = (int32_t)min(t, (long long)INT_MAX);
                c.status[3] += 1;
                *c.ticket = 0;
            }
        }
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = offset_owner(peel_off, c.M, i);
        const int64_t base = m * N;
        const StateIx g = state_ix(c, m);
        int32_t *fn = c.front + (int64_t)nxt * c.M * N + base;
        int32_t *nfn = c.nfront + nxt * c.M + m;
        const int ci = c.cidx[m];
        int32_t *cl = c.cand + (int64_t)ci * c.M * N + base;
        int32_t *ncl = c.ncand + ci * c.M + m;
        const int32_t ep = c.epoch[m];
        const bool cyclic = c.cyc[m] != 0;
        const int32_t v = c.front[(int64_t)cur * c.M * N + base + (i - peel_off[m])];
        const uchar4 mv = c.msk[g(v)];
        const unsigned act = (unsigned)mv.x & ~(unsigned)mv.z;
        const unsigned ob = mv.y;
        int32_t nb[F];
        load_nbr<F>(c, v, nb);
        // all upwind levels in flight together
        int lv[F];
#pragma unroll
        for (int k = 0; k < F; ++k) lv[k] = (((act >> k) & 1u) && nb[k] >= 0) ? st_level(c.st[g(nb[k])]) + 1 : 0;
        int lev = 0;
#pragma unroll
        for (int k = 0; k < F; ++k) lev = max(lev, lv[k]);
        c.st[g(v)] = lev << 4;  // count 0, level set
        // all downwind decrements in flight together
        int32_t old[F];
        // a decrement to zero makes the cell ready; any other one makes it a
        // cycle candidate, once per epoch (stamp).  The stamps are exchanged
        // together with the decrements: a stamp left on a cell that became
        // ready only keeps it out of the candidates, where a walk would drop it.
        int32_t sold[F];
#pragma unroll
        for (int k = 0; k < F; ++k) {
            const bool o = ((ob >> k) & 1u) != 0;
            old[k] = o ? st_count(atomicSub(&c.st[g(nb[k])], 1)) : 0;
            sold[k] = (o && cyclic) ? atomicExch(&c.stamp[g(nb[k])], ep) : ep;
        }
        unsigned rmask = 0, cmask = 0;
#pragma unroll
        for (int k = 0; k < F; ++k)
            if ((ob >> k) & 1u) {
                if (old[k] == 1) rmask |= 1u << k;
                else if (sold[k] != ep) cmask |= 1u << k;
            }
        // list slots: one atomic per list for the lanes of the same direction
        int32_t rb, cb;
        warp_reserve2(nfn, ncl, __popc(rmask), __popc(cmask), (uint64_t)m, rb, cb);
#pragma unroll
        for (int k = 0; k < F; ++k) {
            if ((rmask >> k) & 1u) {
                if (rb < N) fn[rb] = nb[k];
                else atomicCAS(&c.status[0], 0, JSWEEP_ERR_OOM);
                ++rb;
            }
            if ((cmask >> k) & 1u) {
                if (cb < N) cl[cb] = nb[k];
                else atomicCAS(&c.status[0], 0, JSWEEP_ERR_OOM);
                ++cb;
            }
        }
    }
}

// Index of value v in X[0..size), or -1 (warp-cooperative).
__device__ __forceinline__ int warp_find(const int32_t *X, int size, int32_t v, int lane) {
    for (int j0 = 0; j0 < size; j0 += kWarp) {
        int j = j0 + lane;
        unsigned hit = __ballot_sync(0xffffffffu, j < size && X[j] == v);
        if (hit) return j0 + __ffs(hit) - 1;
    }
    return -1;
}

constexpr int kResolveWarps = 16;
constexpr int kSeedCap = 4096;  // cycles kept per direction and step (more wait for the next round)

// Walk from candidate v to the first unfinished active upwind cell (in
// increasing face-slot order), again and again, claiming cells: a cell
// owned (this epoch) by a lower walker id stops the walk, a higher id is taken
// over.  The lowest-id walker that reaches a pointer cycle therefore owns the
// whole cycle and comes back to a cell it owns: that cell is returned (or -1).
// A cell whose count is zero is ready (its upwind cells are all done), so it
// is on no cycle: the walk ends there.  Per cell, the count, the claim word,
// the masks and the neighbours are loaded together, then the upwind levels
// together with the claim's compare-and-swap (levels and counts do not change
// while walks run).
template <int F>
__device__ int32_t claim_walk(const BuildCtx &c, StateIx g, int32_t v, uint32_t me, int32_t ep,
                              int walk_max) {
    const unsigned long long tag = ((unsigned long long)(uint32_t)ep << 32) | me;
    // most candidates are ready by the time of the search: their count alone
    // ends the walk
    if (st_count(c.st[g(v)]) == 0) return -1;
    int32_t x = v;
    for (int step = 0; step < walk_max; ++step) {
        unsigned long long *slot = c.wclaim + g(x);
        const int32_t cx = step == 0 ? 1 : st_count(c.st[g(x)]);
        unsigned long long old = *((volatile unsigned long long *)slot);
        const uchar4 mx = c.msk[g(x)];
        int32_t nb[F];
        load_nbr<F>(c, x, nb);
        if (cx <= 0) return -1;
        const unsigned act = (unsigned)mx.x & ~(unsigned)mx.z;
        int lv[F];
#pragma unroll
        for (int k = 0; k < F; ++k) lv[k] = (((act >> k) & 1u) && nb[k] >= 0) ? st_level(c.st[g(nb[k])]) : 0;
        while (true) {
            if ((int32_t)(old >> 32) == ep) {
                const uint32_t owner = (uint32_t)old;
                if (owner == me) return x;  // closed a cycle of our own
                if (owner < me) return -1;  // a lower walker owns this path
            }
            const unsigned long long prev = atomicCAS(slot, old, tag);
            if (prev == old) break;
            old = prev;
        }
        // first unfinished active upwind cell (slots in increasing face id)
        int32_t p = -1;
#pragma unroll
        for (int k = F - 1; k >= 0; --k)
            if (((act >> k) & 1u) && nb[k] >= 0 && lv[k] < 0) p = nb[k];
        if (p < 0) return -1;
        x = p;
    }
    return -1;
}

// Cycle resolution runs in every unfinished direction that has stalled and,
// in an eager search, also in every one that is not certified acyclic and has
// new candidates.  A component is then resolved as soon as a walk can close
// it, not only when the whole direction has stalled, so that the cells behind
// it are not held back until the rest of the front drains.  The closure test
// only ever accepts a set closed under unfinished upwind cells, which contains
// the whole component whatever the frontier holds.
__device__ __forceinline__ bool resolve_active(const BuildCtx &c, int64_t m, int nxt, bool eager, bool *stalled) {
    if (c.nproc[m] >= c.N) return false;  // direction finished
    *stalled = c.nfront[nxt * c.M + m] == 0;
    return *stalled || (eager && c.cyc[m] != 0 && c.ncand[c.cidx[m] * c.M + m] != 0);
}

// Walks (grid (blocks, direction)): every thread walks candidates with
// claim_walk and records the cells at which it closed a pointer cycle.
template <int F>
__global__ void k_walk(BuildCtx c, int nxt, int eager, int walk_max) {
    const int64_t m = blockIdx.y;
    bool stalled;
    if (!resolve_active(c, m, nxt, eager != 0, &stalled)) return;
    const int64_t base = m * c.N;
    const StateIx g = state_ix(c, m);
    const int ci = c.cidx[m];
    const int32_t nc = min(c.ncand[ci * c.M + m], (int32_t)c.N);
    const int32_t *cl = c.cand + (int64_t)ci * c.M * c.N + base;
    const int32_t ep = c.epoch[m];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
        // a finished or ready candidate (count zero) ends its walk at once
        const int32_t x = claim_walk<F>(c, g, cl[i], (uint32_t)i + 1u, ep, walk_max);
        if (x >= 0) {
            const int32_t k = atomicAdd(&c.nseeds[m], 1);
            if (k < kSeedCap) c.seeds[m * kSeedCap + k] = x;
        }
    }
}

// Closures (blockIdx.x = direction): one warp per recorded cycle gathers the
// unfinished cells that reach it backwards (cap B); when that set closes, the
// cycle's strongly connected component is computed inside it and its smallest
// active face is lagged (one lag per component: the component is claimed
// through its smallest cell).  Then the direction's candidate lists are
// rotated.  Dynamic shared memory: per warp X[B] (int32), Sidx[B] (int32),
// inS[B] (uint8).
__global__ void __launch_bounds__(kResolveWarps * 32, 2) k_resolve(BuildCtx c, int nxt, int eager, int B, int Beager) {
    const int64_t m = blockIdx.x;
    bool stalled;
    if (!resolve_active(c, m, nxt, eager != 0, &stalled)) return;
    extern __shared__ int32_t sh[];
    __shared__ int32_t new_lags;
    const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
    if (threadIdx.x == 0) new_lags = 0;
    __syncthreads();
    const int64_t base = m * c.N;
    const StateIx g = state_ix(c, m);
    const int ci = c.cidx[m];
    const int32_t nc = min(c.ncand[ci * c.M + m], (int32_t)c.N);
    const int32_t *cl = c.cand + (int64_t)ci * c.M * c.N + base;
    int32_t *cn = c.cand + (int64_t)(ci ^ 1) * c.M * c.N + base;
    int32_t *ncn = c.ncand + (ci ^ 1) * c.M + m;
    const int32_t ep = c.epoch[m];
    const int32_t nseeds = c.nseeds[m];
    const int ns_total = min(nseeds, kSeedCap);
    const int32_t *seeds = c.seeds + m * kSeedCap;
    if (threadIdx.x == 0) atomicAdd(&c.status[5], ns_total);

    int32_t *X = sh + warp * (2 * B + (B + 3) / 4);
    int32_t *Sidx = X + B;
    uint8_t *inS = reinterpret_cast<uint8_t *>(Sidx + B);
    int my_lags = 0;
    // Before a direction stalls, the backward closure of a cycle often runs into
    // upstream cells that are merely not peeled yet and cannot close; an eager
    // search therefore stops at Beager cells, a stalled direction searches up
    // to B.  A closure that does not close is retried later, so the lags found
    // do not depend on the caps (only whether the build succeeds can).
    const int Bcap = stalled ? B : min(B, Beager);
    for (int si = warp; si < ns_total; si += kResolveWarps) {
        const int32_t seed = seeds[si];
        // ---- backward closure of the seed over unfinished cells, capped at B.
        // Breadth first: the lanes take up to 32 cells of the current front at
        // once (their loads in flight together); new cells are appended one by
        // one (shared memory only).  Whether the closure fits under the cap
        // does not depend on the order cells are found in.
        if (lane == 0) X[0] = seed;
        __syncwarp();
        int size = 1, head = 0;
        bool closed = true;
        while (head < size && closed) {
            const int nfr = min(size - head, kWarp);
            int32_t up[kMaxFaces];
            unsigned upm = 0;
            if (lane < nfr) {
                const int32_t x = X[head + lane];
                const uchar4 mx = c.msk[g(x)];
                const unsigned act = (unsigned)mx.x & ~(unsigned)mx.z;
                int lv[kMaxFaces];
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k)
                    up[k] = (k < c.FS && ((act >> k) & 1u)) ? c.nbr[(int64_t)x * c.FS + k] : -1;
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k) lv[k] = up[k] >= 0 ? st_level(c.st[g(up[k])]) : 0;
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k)
                    if (up[k] >= 0 && lv[k] < 0) upm |= 1u << k;
            }
            head += nfr;
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k) {
                unsigned todo = __ballot_sync(0xffffffffu, (upm >> k) & 1u);
                while (todo && closed) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const int32_t uu = __shfl_sync(0xffffffffu, up[k], src);
                    if (warp_find(X, size, uu, lane) < 0) {
                        if (size == Bcap) {
                            closed = false;
                        } else {
                            if (lane == 0) X[size] = uu;
                            __syncwarp();
                            ++size;
                        }
                    }
                }
            }
        }
        if (!closed) continue;

        // ---- strongly connected component of the seed inside the closure:
        // every cell of X reaches the seed, so the cells reached from the seed
        // within X form its component (breadth first, lanes over the front).
        for (int j = lane; j < size; j += kWarp) inS[j] = 0;
        __syncwarp();
        if (lane == 0) {
            inS[0] = 1;
            Sidx[0] = 0;
        }
        __syncwarp();
        int ns = 1, h = 0;
        while (h < ns) {
            const int nfr = min(ns - h, kWarp);
            int32_t dn[kMaxFaces];
            unsigned dnm = 0;
            if (lane < nfr) {
                const int32_t y = X[Sidx[h + lane]];
                const unsigned ob = c.msk[g(y)].y;
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k) {
                    dn[k] = (k < c.FS && ((ob >> k) & 1u)) ? c.nbr[(int64_t)y * c.FS + k] : -1;
                    if (dn[k] >= 0) dnm |= 1u << k;
                }
            }
            __syncwarp();
            h += nfr;
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k) {
                unsigned todo = __ballot_sync(0xffffffffu, (dnm >> k) & 1u);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const int32_t ww = __shfl_sync(0xffffffffu, dn[k], src);
                    const int j = warp_find(X, size, ww, lane);
                    if (j >= 0 && !inS[j]) {
                        __syncwarp();
                        if (lane == 0) {
                            inS[j] = 1;
                            Sidx[ns] = j;
                        }
                        __syncwarp();
                        ++ns;
                    }
                }
            }
        }
        if (ns < 2) continue;

        // ---- smallest active face inside the component (each face is the
        // outgoing face of exactly one of its cells, so the minimum is unique),
        // and the component's smallest cell; lanes load 32 cells at once
        int32_t best_f = INT_MAX, best_u = -1, best_v = -1, smin = INT_MAX;
        for (int t0 = 0; t0 < ns; t0 += kWarp) {
            int32_t dn[kMaxFaces], fk[kMaxFaces];
            unsigned dnm = 0;
            int32_t y = -1;
            if (t0 + lane < ns) {
                y = X[Sidx[t0 + lane]];
                smin = min(smin, y);
                const unsigned ob = c.msk[g(y)].y;
#pragma unroll
                for (int k = 0; k < kMaxFaces; ++k) {
                    const bool o = k < c.FS && ((ob >> k) & 1u);
                    dn[k] = o ? c.nbr[(int64_t)y * c.FS + k] : -1;
                    fk[k] = o ? (c.sface[(int64_t)y * c.FS + k] >> 1) : INT_MAX;
                    if (dn[k] >= 0) dnm |= 1u << k;
                }
            }
#pragma unroll
            for (int k = 0; k < kMaxFaces; ++k) {
                unsigned todo = __ballot_sync(0xffffffffu, (dnm >> k) & 1u);
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const int32_t ww = __shfl_sync(0xffffffffu, dn[k], src);
                    const int32_t ff = __shfl_sync(0xffffffffu, fk[k], src);
                    const int32_t yy = __shfl_sync(0xffffffffu, y, src);
                    const int j = warp_find(X, size, ww, lane);
                    if (j >= 0 && inS[j] && ff < best_f) {
                        best_f = ff;
                        best_u = yy;
                        best_v = ww;
                    }
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
        // ---- one warp per component records the lag (claimed by its smallest cell)
        if (lane == 0 && best_f != INT_MAX) {
            if (atomicExch(&c.claim[g(smin)], ep) != ep) {
                int32_t k = atomicAdd(c.npend, 1);
                if (k < c.pend_cap) {
                    c.pend[k] = make_int4((int)m, best_f, best_u, best_v);
                    ++my_lags;
                } else {
                    atomicCAS(&c.status[0], 0, JSWEEP_ERR_OOM);
                }
            } else {
                best_f = INT_MAX;  // someone else owns this component
            }
        }
        best_f = __shfl_sync(0xffffffffu, best_f, 0);
        if (best_f != INT_MAX) {
            // members become candidates of the next stall
            for (int t = lane; t < ns; t += kWarp) {
                int32_t y = X[Sidx[t]];
                if (atomicExch(&c.stamp[g(y)], ep + 1) != ep + 1) push(cn, ncn, y, c.N, c.status);
            }
        }
        __syncwarp();
    }
    if (lane == 0 && my_lags) atomicAdd(&new_lags, my_lags);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&c.status[4], 1);
        atomicAdd(&c.status[6], new_lags);
        if (stalled && new_lags == 0 && nseeds <= kSeedCap) {
            // stalled and nothing found: a component larger than the search cap
            if (atomicCAS(&c.status[0], 0, JSWEEP_ERR_CYCLE) == 0) c.status[1] = (int32_t)m;
        }
        if (nseeds > kSeedCap) {
            // seeds were dropped: keep this round's candidates for the next stall
            for (int32_t i = 0; i < nc; ++i) {
                int32_t v = cl[i];
                if (c.st[g(v)] < 0 && atomicExch(&c.stamp[g(v)], ep + 1) != ep + 1) push(cn, ncn, v, c.N, c.status);
            }
        }
        c.ncand[ci * c.M + m] = 0;
        c.cidx[m] = ci ^ 1;
        c.epoch[m] = ep + 1;
        c.nseeds[m] = 0;
    }
}

__device__ __forceinline__ int slot_of(const BuildCtx &c, int32_t cell, int32_t f) {
    for (int k = 0; k < c.FS; ++k)
        if ((c.sface[(int64_t)cell * c.FS + k] >> 1) == f) return k;
    return -1;
}

// Applies the lags of a cycle search (the pending list is cleared by the next
// step's peel, after every block here has read its length).
__global__ void k_commit(BuildCtx c, int nxt) {
    const int32_t n = min(*c.npend, (int32_t)c.pend_cap);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int4 e = c.pend[i];
        int64_t m = e.x;
        int32_t f = e.y, up = e.z, dn = e.w;
        int64_t base = m * c.N;
        const StateIx g = state_ix(c, m);
        int kd = slot_of(c, dn, f), ku = slot_of(c, up, f);
        if (kd < 0 || ku < 0) {
            atomicCAS(&c.status[0], 0, JSWEEP_ERR_CYCLE);
            continue;
        }
        c.msk[g(dn)].z |= (uint8_t)(1u << kd);
        c.msk[g(up)].y &= (uint8_t)~(1u << ku);
        const int32_t old = st_count(atomicSub(&c.st[g(dn)], 1));
        if (old == 1) push(c.front + (int64_t)nxt * c.M * c.N + base, c.nfront + nxt * c.M + m, dn, c.N, c.status);
        int32_t k = atomicAdd(c.nlag, 1);
        if (k < c.lag_cap) c.lagall[k] = e; else atomicCAS(&c.status[0], 0, JSWEEP_ERR_OOM);
    }
}

// State words [S / 8][N][8] back to [M][N] (sdir[s] = direction of slot s, or -1
// for a padding slot): one thread reads a cell's 8 slots (32 bytes).  LEVEL:
// the words are frontier-loop state words and the level is stored.
template <bool LEVEL>
__global__ void k_ungroup(const uint32_t *src, const int32_t *sdir, int64_t N, int64_t S, uint32_t *dst) {
    const int64_t n = S / 8 * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gi = i / N, v = i - gi * N;
        const uint4 a = reinterpret_cast<const uint4 *>(src)[2 * i], b = reinterpret_cast<const uint4 *>(src)[2 * i + 1];
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int32_t m = __ldg(sdir + gi * 8 + j);
            if (m >= 0) dst[m * N + v] = LEVEL ? (uint32_t)st_level((int32_t)w[j]) : w[j];
        }
    }
}

__global__ void k_level_max(const int32_t *lvl, int64_t N, int64_t M, int32_t *lmax) {
    int64_t m = blockIdx.y;
    int best = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        best = max(best, lvl[m * N + i]);
    for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
    if ((threadIdx.x & 31) == 0) atomicMax(&lmax[m], best);
}

// level_ptr of direction m from its sorted keys.
__global__ void k_level_ptr(const uint32_t *skeys, int64_t N, int64_t M, const int64_t *lp_off,
                            const int32_t *nlev, int32_t *lp) {
    int64_t m = blockIdx.y;
    int32_t *out = lp + lp_off[m];
    const uint32_t *k = skeys + m * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t prev = i == 0 ? 0xffffffffu : k[i - 1];
        uint32_t cur = k[i];
        if (i == 0 || cur != prev) {
            uint32_t lo = i == 0 ? 0u : prev + 1;
            for (uint32_t l = lo; l <= cur; ++l) out[l] = (int32_t)i;
        }
        if (i == N - 1) out[nlev[m]] = (int32_t)N;
    }
}

__global__ void k_mask_level_order(const uchar4 *msk, const int32_t *order, int64_t N, int64_t M, uint8_t *mask) {
    const int64_t total = N * M;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = idx / N;
        int32_t c = order[idx];
        int64_t src = m * N + c;
        const uchar4 ms = msk[src];
        mask[idx] = (uint8_t)(ms.x | (ms.z ? 0x80u : 0u));
    }
}

__global__ void k_lag_keys(const int4 *lagall, int32_t T, uint32_t *kf, uint32_t *km) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        kf[i] = (uint32_t)lagall[i].y;
        km[i] = (uint32_t)lagall[i].x;
    }
}

__global__ void k_gather_u32(const uint32_t *src, const int32_t *perm, int32_t n, uint32_t *dst) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = src[perm[i]];
}

__global__ void k_lag_scatter(const int4 *lagall, const int32_t *perm, int32_t T, int32_t *lm,
                              int32_t *lf, int32_t *lu, int32_t *ld) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
        int4 e = lagall[perm[i]];
        lm[i] = e.x;
        lf[i] = e.y;
        lu[i] = e.z;
        ld[i] = e.w;
    }
}

__global__ void k_lag_ptr(const int32_t *lm, int32_t T, int64_t M, int32_t *lag_ptr) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= T; i += gridDim.x * blockDim.x) {
        int32_t prev = i == 0 ? -1 : lm[i - 1];
        int32_t cur = i == T ? (int32_t)M : lm[i];
        for (int32_t mm = prev + 1; mm <= cur; ++mm) lag_ptr[mm] = i;
    }
}

// Octant-aligned schedule layers (blockIdx.x = direction m):
// kappa(c) = max(floor(rho_o * lambda_o(c)), 1 + max kappa(active upwind cell)).
// Upwind cells have smaller levels, so their kappa is final when c's level runs;
// one block sweeps its direction level after level with a block barrier in
// between (a direction's levels need no other direction).
__global__ void __launch_bounds__(1024)
    k_kappa_dir(const int32_t *order, const int32_t *lp, const int64_t *lp_off, const int32_t *nlev,
                const uchar4 *msk, const int4 *nbr8, int64_t N, const int32_t *oct,
                const float *rho, const int32_t *lam, int32_t *kap) {
    const int64_t m = blockIdx.x;
    const int o = oct[m];
    const float r = rho[o];
    const int64_t base = m * N;
    const int L = nlev[m];
    const int32_t *lpm = lp + lp_off[m];
    for (int l = 0; l < L; ++l) {
        const int32_t p0 = lpm[l], p1 = lpm[l + 1];
        for (int32_t pos = p0 + threadIdx.x; pos < p1; pos += blockDim.x) {
            const int32_t c = order[base + pos];
            int32_t k = (int32_t)(r * (float)lam[(int64_t)o * N + c]);
            const uchar4 mc = msk[base + c];
            const unsigned act = (unsigned)mc.x & ~(unsigned)mc.z;
            const int4 a = __ldg(nbr8 + 2 * (int64_t)c), b = __ldg(nbr8 + 2 * (int64_t)c + 1);
            const int32_t nb[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            int32_t kk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) kk[q] = (((act >> q) & 1u) && nb[q] >= 0) ? __ldcg(kap + base + nb[q]) + 1 : k;
#pragma unroll
            for (int q = 0; q < 8; ++q) k = max(k, kk[q]);
            kap[base + c] = k;
        }
        __syncthreads();  // this level's layers are stored before the next level reads them
    }
}

// ---- exclusive scan of int64 (three-phase, recursive over block sums) ------------
constexpr int kScanThreads = 1024, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__device__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int64_t before = warp ? wsum[warp - 1] : 0;
    if (total) *total = wsum[(blockDim.x >> 5) - 1];
    int64_t r = before + x - v;
    __syncthreads();
    return r;
}

__global__ void k_scan_sums(const int64_t *in, int64_t n, int64_t *sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int64_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int64_t *in, int64_t n, const int64_t *offs, int64_t *out) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        s += v[k];
    }
    int64_t pre = block_exclusive_scan(s, nullptr) + (offs ? offs[blockIdx.x] : 0);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
}

// ---- stable LSD radix sort of equal-length segments (8-bit digits) -----------------
// A block sorts one tile of kRsTile keys per pass: each of its warps loads its
// kRsWarpKeys keys into registers at once (all loads in flight together), the
// tile's digit counts go to a [256][tiles] histogram, and after its scan each
// warp ranks its keys in order (lanes with equal digits by __match_any_sync),
// starting where the earlier tiles and the block's earlier warps end: the
// order of equal digits is the order of the input (stable).
constexpr int kRsWarps = 4;                       // warps per block
constexpr int kRsWarpKeys = 1024;                 // keys per warp, 32 per lane
constexpr int kRsTile = kRsWarps * kRsWarpKeys;   // keys per block tile
constexpr int kRsPerLane = kRsWarpKeys / 32;
__global__ void __launch_bounds__(kRsWarps * 32)
    k_rs_hist(const uint32_t *keys, int64_t seg_len, int shift, int32_t *hist, int64_t tiles) {
    __shared__ int32_t hs[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t s = blockIdx.y, t = blockIdx.x;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hs[b] = 0;
    __syncthreads();
    const int64_t e0 = t * kRsTile + (int64_t)w * kRsWarpKeys;  // first key of this warp in the segment
    const int64_t rem = seg_len - e0;
    uint32_t kr[kRsPerLane];
#pragma unroll
    for (int i = 0; i < kRsPerLane; ++i) kr[i] = i * 32 + lane < rem ? __ldg(keys + s * seg_len + e0 + i * 32 + lane) : 0u;
#pragma unroll
    for (int i = 0; i < kRsPerLane; ++i)
        if (i * 32 + lane < rem) atomicAdd(&hs[(kr[i] >> shift) & 255u], 1);
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[(s * 256 + b) * tiles + t] = hs[b];
}

// In-place exclusive scan of each segment's [256][tiles] histogram (one block
// per segment, four entries per thread and round; len is a multiple of 256).
__global__ void k_rs_scan(int32_t *hist, int64_t len) {
    int4 *h = reinterpret_cast<int4 *>(hist + blockIdx.x * len);
    const int64_t n4 = len / 4;
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n4; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int4 v = i < n4 ? h[i] : make_int4(0, 0, 0, 0);
        int64_t tot;
        const int64_t ex = block_exclusive_scan((int64_t)v.x + v.y + v.z + v.w, &tot);
        int64_t p = carry + ex;
        if (i < n4) {
            int4 o;
            o.x = (int32_t)p;
            p += v.x;
            o.y = (int32_t)p;
            p += v.y;
            o.z = (int32_t)p;
            p += v.z;
            o.w = (int32_t)p;
            h[i] = o;
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

// VALS: values come from vals[]; otherwise a key's value is its index in the segment.
template <bool VALS>
__global__ void __launch_bounds__(kRsWarps * 32)
    k_rs_scatter(const uint32_t *keys, const int32_t *vals, int64_t seg_len, int shift, const int32_t *hist,
                 int64_t tiles, uint32_t *keys_out, int32_t *vals_out) {
    __shared__ int32_t runs[kRsWarps][256];  // this warp's digit counts, then its next position per digit
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t s = blockIdx.y, t = blockIdx.x;
    int32_t *run = runs[w];
    for (int b = lane; b < 256; b += 32) run[b] = 0;
    const int64_t e0 = t * kRsTile + (int64_t)w * kRsWarpKeys;
    const int64_t rem = seg_len - e0;
    uint32_t kr[kRsPerLane];
    int32_t vr[VALS ? kRsPerLane : 1];
#pragma unroll
    for (int i = 0; i < kRsPerLane; ++i) kr[i] = i * 32 + lane < rem ? __ldg(keys + s * seg_len + e0 + i * 32 + lane) : 0u;
    if constexpr (VALS) {
#pragma unroll
        for (int i = 0; i < kRsPerLane; ++i) vr[i] = i * 32 + lane < rem ? __ldg(vals + s * seg_len + e0 + i * 32 + lane) : 0;
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kRsPerLane; ++i)
        if (i * 32 + lane < rem) atomicAdd(&run[(kr[i] >> shift) & 255u], 1);
    __syncthreads();
    // a warp's run of digit b starts after the tile's earlier tiles and earlier warps
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        int32_t p = hist[(s * 256 + b) * tiles + t];
#pragma unroll
        for (int w2 = 0; w2 < kRsWarps; ++w2) {
            const int32_t c = runs[w2][b];
            runs[w2][b] = p;
            p += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsPerLane; ++i) {
        const bool valid = i * 32 + lane < rem;
        const uint32_t key = kr[i];
        const unsigned d = valid ? ((key >> shift) & 255u) : (256u + lane);
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lanemask_lt());
        const int pos = valid ? run[d] + rank : 0;
        __syncwarp();
        if (valid && rank == 0) run[d] += __popc(peers);
        __syncwarp();
        if (valid) {
            int32_t val;
            if constexpr (VALS) val = vr[i];
            else val = (int32_t)(e0 + i * 32 + lane);
            if (keys_out) keys_out[s * seg_len + pos] = key;
            vals_out[s * seg_len + pos] = val;
        }
    }
}

}  // namespace

int scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n <= 0) return JSWEEP_OK;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_apply<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        JS_LAUNCH_CHECK();
        return JSWEEP_OK;
    }
    DevBuf sums, offs;
    JS_TRY(sums.alloc(nb * 8, s));
    JS_TRY(offs.alloc(nb * 8, s));
    k_scan_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums.as<int64_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(scan_exclusive_i64(sums.as<int64_t>(), offs.as<int64_t>(), nb, s));
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, offs.as<int64_t>(), out);
    JS_LAUNCH_CHECK();
    JS_CUDA(cudaStreamSynchronize(s));  // sums/offs are released on return
    return JSWEEP_OK;
}

int radix_sort_segments(const uint32_t *keys_in, int64_t n_seg, int64_t seg_len, int key_bits,
                        const int32_t *vals_in, int32_t *vals_out, uint32_t *keys_out,
                        cudaStream_t s) {
    if (n_seg <= 0 || seg_len <= 0) return JSWEEP_OK;
    const int64_t tiles = (seg_len + kRsTile - 1) / kRsTile;
    int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
    DevBuf hist, kb[2], vb[2];
    JS_TRY(hist.alloc((size_t)n_seg * 256 * tiles * 4, s));
    size_t ne = (size_t)n_seg * seg_len;
    // passes before the last ping-pong between scratch buffers; the last one
    // writes the outputs (keys only where asked for)
    for (int b = 0; b < std::min(passes - 1, 2); ++b) {
        JS_TRY(kb[b].alloc(ne * 4, s));
        JS_TRY(vb[b].alloc(ne * 4, s));
    }
    const uint32_t *kin = keys_in;
    const int32_t *vin = vals_in;
    dim3 grid((unsigned)tiles, (unsigned)n_seg);
    for (int p = 0; p < passes; ++p) {
        const bool last = p == passes - 1;
        uint32_t *ko = last ? keys_out : kb[p & 1].as<uint32_t>();
        int32_t *vo = last ? vals_out : vb[p & 1].as<int32_t>();
        k_rs_hist<<<grid, kRsWarps * 32, 0, s>>>(kin, seg_len, 8 * p, hist.as<int32_t>(), tiles);
        JS_LAUNCH_CHECK();
        k_rs_scan<<<(unsigned)n_seg, 1024, 0, s>>>(hist.as<int32_t>(), 256 * tiles);
        JS_LAUNCH_CHECK();
        if (vin)
            k_rs_scatter<true><<<grid, kRsWarps * 32, 0, s>>>(kin, vin, seg_len, 8 * p, hist.as<int32_t>(), tiles, ko, vo);
        else
            k_rs_scatter<false><<<grid, kRsWarps * 32, 0, s>>>(kin, vin, seg_len, 8 * p, hist.as<int32_t>(), tiles, ko, vo);
        JS_LAUNCH_CHECK();
        kin = ko;
        vin = vo;
    }
    JS_CUDA(cudaStreamSynchronize(s));
    return JSWEEP_OK;
}

// Octant of every direction: bits (1, 2, 4) set for negative (x, y, z).
static std::vector<int32_t> octant_of(const Dags *d) {
    std::vector<int32_t> oct(d->M);
    for (int64_t m = 0; m < d->M; ++m) {
        const double *o = d->quad->dirs.data() + 3 * m;
        oct[m] = (o[0] < 0 ? 1 : 0) | (o[1] < 0 ? 2 : 0) | (o[2] < 0 ? 4 : 0);
    }
    return oct;
}

// State slots of the frontier loop: the directions of each octant in index
// order get consecutive slots; an octant's run is padded to a multiple of 8
// when that costs at most half as many slots as it has directions (a lone
// diagonal is not).  Returns S (a multiple of 8); sdir[s] = direction or -1.
static int64_t state_slots(const std::vector<int32_t> &oct, std::vector<int32_t> &dslot, std::vector<int32_t> &sdir) {
    const int64_t M = (int64_t)oct.size();
    dslot.assign(M, -1);
    int64_t S = 0;
    for (int o = 0; o < 8; ++o) {
        int64_t count = 0;
        for (int64_t m = 0; m < M; ++m)
            if (oct[m] == o) {
                dslot[m] = (int32_t)S++;
                ++count;
            }
        const int64_t pad = (8 - S % 8) % 8;
        if (count > 0 && 2 * pad <= count) S += pad;
    }
    S = (S + 7) / 8 * 8;
    sdir.assign(S, -1);
    for (int64_t m = 0; m < M; ++m) sdir[dslot[m]] = (int32_t)m;
    return S;
}

// Dependency graphs of the 8 octant diagonals (+-1, +-1, +-1)/sqrt(3) over the
// same mesh (a nested build with longest-path levels).  Returns nullptr (and no
// error) if that build fails: the diagonals only serve the schedule.
Dags *build_diagonals(Dags *d, cudaStream_t s) {
    Quad *dq = new Quad();
    dq->M = 8;
    std::vector<double> dd(24), dw(8, 1.0);
    const double inv = 1.0 / std::sqrt(3.0);
    for (int o = 0; o < 8; ++o) {
        dd[3 * o] = (o & 1) ? -inv : inv;
        dd[3 * o + 1] = (o & 2) ? -inv : inv;
        dd[3 * o + 2] = (o & 4) ? -inv : inv;
    }
    dq->dirs = dd;
    dq->w = dw;
    if (dq->dirs64.alloc(24 * 8, s) != JSWEEP_OK ||
        cudaMemcpy(dq->dirs64.p, dd.data(), 24 * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete dq;
        clear_error();
        return nullptr;
    }
    Dags *dg = new Dags();
    dg->mesh = d->mesh;
    d->mesh->refs.fetch_add(1);
    dg->quad = dq;  // owned by dg
    dg->N = d->N;
    dg->M = 8;
    dg->opt = d->opt;
    dg->opt.layering = JSWEEP_LAYERS_LEVEL;
    if (build_dags(dg, s) != JSWEEP_OK) {
        delete dg;
        clear_error();
        return nullptr;
    }
    return dg;
}

// Octant-aligned schedule layers (see jsweep_options.layering) from the levels
// of the octant diagonals.
static int octant_layers(Dags *d, const Dags *dg, const std::vector<int32_t> &oct, const uchar4 *msk,
                         const int64_t *lpoff_dev, const int32_t *nlev_dev, cudaStream_t s) {
    const int64_t N = d->N, M = d->M;
    std::vector<float> rho(8, 1.0f);
    for (int o = 0; o < 8; ++o) {
        int64_t lmax = 0;
        for (int64_t m = 0; m < M; ++m)
            if (oct[m] == o) lmax = std::max(lmax, d->nlevels[m]);
        if (lmax > 0) rho[o] = (float)((double)lmax / (double)dg->nlevels[o]);
    }
    DevBuf oct_d, rho_d, kap, skeys, kmax;
    JS_TRY(oct_d.alloc(M * 4, s));
    JS_TRY(rho_d.alloc(8 * 4, s));
    JS_TRY(kap.alloc(N * M * 4, s));
    JS_CUDA(cudaMemcpyAsync(oct_d.p, oct.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(rho_d.p, rho.data(), 8 * 4, cudaMemcpyHostToDevice, s));
    k_kappa_dir<<<(unsigned)M, 1024, 0, s>>>(d->order.as<int32_t>(), d->lp.as<int32_t>(), lpoff_dev, nlev_dev, msk,
                                             d->mesh->nbr8.as<int4>(), N, oct_d.as<int32_t>(),
                                             rho_d.as<float>(), dg->level.as<int32_t>(), kap.as<int32_t>());
    JS_LAUNCH_CHECK();
    // layer counts, sort by (layer, cell id), layer pointers, mask in layer order
    JS_TRY(kmax.alloc(M * 4, s));
    JS_CUDA(cudaMemsetAsync(kmax.p, 0xff, M * 4, s));
    k_level_max<<<dim3(std::min<int64_t>(64, (N + 255) / 256), (unsigned)M), 256, 0, s>>>(kap.as<int32_t>(), N, M,
                                                                                         kmax.as<int32_t>());
    JS_LAUNCH_CHECK();
    std::vector<int32_t> km(M);
    JS_CUDA(cudaMemcpyAsync(km.data(), kmax.p, M * 4, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> nl(M), off(M + 1, 0);
    int64_t smax = 0;
    for (int64_t m = 0; m < M; ++m) {
        nl[m] = (int64_t)km[m] + 1;
        smax = std::max(smax, nl[m]);
        off[m + 1] = off[m] + nl[m] + 1;
    }
    if (smax >= (1ll << 24)) return JSWEEP_OK;  // keep levels
    int key_bits = 1;
    while ((1ll << key_bits) < smax) ++key_bits;
    JS_TRY(d->korder.alloc(N * M * 4, s));
    JS_TRY(skeys.alloc(N * M * 4, s));
    JS_TRY(radix_sort_segments(reinterpret_cast<const uint32_t *>(kap.p), M, N, key_bits, nullptr,
                               d->korder.as<int32_t>(), skeys.as<uint32_t>(), s));
    DevBuf off_d, nl_d;
    std::vector<int32_t> nl32(M);
    for (int64_t m = 0; m < M; ++m) nl32[m] = (int32_t)nl[m];
    JS_TRY(off_d.alloc((M + 1) * 8, s));
    JS_TRY(nl_d.alloc(M * 4, s));
    JS_CUDA(cudaMemcpyAsync(off_d.p, off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nl_d.p, nl32.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(d->klp.alloc(off[M] * 4, s));
    k_level_ptr<<<dim3(std::min<int64_t>(64, (N + 255) / 256), (unsigned)M), 256, 0, s>>>(
        skeys.as<uint32_t>(), N, M, off_d.as<int64_t>(), nl_d.as<int32_t>(), d->klp.as<int32_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(d->kmask.alloc(N * M, s));
    k_mask_level_order<<<grid_for(N * M, 256, 152 * 64), 256, 0, s>>>(msk, d->korder.as<int32_t>(), N, M,
                                                                      d->kmask.as<uint8_t>());
    JS_LAUNCH_CHECK();
    JS_CUDA(cudaStreamSynchronize(s));
    d->layering = JSWEEP_LAYERS_OCTANT;
    d->s_order = d->korder.as<int32_t>();
    d->s_mask = d->kmask.as<uint8_t>();
    d->s_lp = d->klp.as<int32_t>();
    d->slayers = nl;
    d->sp_off = off;
    d->Smax = smax;
    return JSWEEP_OK;
}

int build_dags(Dags *d, cudaStream_t s) {
    Mesh *mesh = d->mesh;
    Quad *quad = d->quad;
    const int64_t N = d->N, M = d->M, MN = N * M;
    if (!d->ev[0])
        for (auto &e : d->ev) JS_CUDA(cudaEventCreate(&e));
    JS_CUDA(cudaEventRecord(d->ev[0], s));
    // phase boundaries (device time of each build phase)
    cudaEvent_t pe[7];
    for (auto &e : pe) JS_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 7; ++i) cudaEventDestroy(e[i]);
        }
    } ev_guard{pe};
    for (int i = 0; i < 6; ++i) d->timing.build_phase_ms[i] = 0.0;

    // ---- scratch (per-(direction, cell) state in slot-grouped layout, SN words)
    std::vector<int32_t> oct = octant_of(d);
    std::vector<int32_t> dslot, sdir;
    const int64_t S = state_slots(oct, dslot, sdir), SN = S * N;
    DevBuf st_g, stamp, claim, wclaim, msk_g, front, cand, small, pend, lagall, dslot_d, sdir_d;
    JS_TRY(st_g.alloc(SN * 4, s));
    JS_TRY(stamp.alloc(SN * 4, s));
    JS_TRY(claim.alloc(SN * 4, s));
    JS_TRY(wclaim.alloc(SN * 8, s));
    JS_TRY(msk_g.alloc(SN * 4, s));
    JS_TRY(dslot_d.alloc(M * 4, s));
    JS_TRY(sdir_d.alloc(S * 4, s));
    JS_CUDA(cudaMemcpyAsync(dslot_d.p, dslot.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(sdir_d.p, sdir.data(), S * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(front.alloc(2 * MN * 4, s));
    JS_TRY(cand.alloc(2 * MN * 4, s));
    // small: nfront[2M] ncand[2M] cidx[M] epoch[M] nproc[M] npend nlag status[4]
    const int64_t n_small = 7 * M + 16;
    JS_TRY(small.alloc(n_small * 4, s));
    const int64_t pend_cap = std::max<int64_t>(1 << 16, std::min<int64_t>(MN, 1 << 22));
    const int64_t lag_cap = std::max<int64_t>(1 << 16, std::min<int64_t>(MN, std::max<int64_t>(1 << 20, MN / 64)));
    JS_TRY(pend.alloc(pend_cap * 16, s));
    JS_TRY(lagall.alloc(lag_cap * 16, s));

    BuildCtx c;
    c.N = N;
    c.M = M;
    c.FS = mesh->FS;
    c.sface = mesh->sface.as<int32_t>();
    c.nbr = mesh->nbr.as<int32_t>();
    c.nbr8 = mesh->nbr8.as<int4>();
    c.normal = mesh->normal.as<double>();
    c.dirs = quad->dirs64.as<double>();
    c.st = st_g.as<int32_t>();
    c.stamp = stamp.as<int32_t>();
    c.claim = claim.as<int32_t>();
    c.wclaim = wclaim.as<unsigned long long>();
    c.msk = msk_g.as<uchar4>();
    c.dslot = dslot_d.as<int32_t>();
    c.sdir = sdir_d.as<int32_t>();
    c.S = S;
    c.front = front.as<int32_t>();
    c.cand = cand.as<int32_t>();
    int32_t *sm = small.as<int32_t>();
    c.nfront = sm;
    c.ncand = sm + 2 * M;
    c.cidx = sm + 4 * M;
    c.epoch = sm + 5 * M;
    c.nproc = sm + 6 * M;
    c.npend = sm + 7 * M;
    c.nlag = sm + 7 * M + 1;
    c.status = sm + 7 * M + 4;
    c.ticket = sm + 7 * M + 12;
    c.pend = pend.as<int4>();
    c.pend_cap = pend_cap;
    c.lagall = lagall.as<int4>();
    c.lag_cap = lag_cap;

    // masks, state words, stamps and claims: every word is written by k_classify
    JS_CUDA(cudaMemsetAsync(sm, 0, n_small * 4, s));
    {
        std::vector<int32_t> ones(M, 1);
        JS_CUDA(cudaMemcpyAsync(c.epoch, ones.data(), M * 4, cudaMemcpyHostToDevice, s));
        JS_CUDA(cudaStreamSynchronize(s));
    }
    // diagonals of the octants first: their levels certify acyclic directions and
    // give the octant-aligned schedule layers
    DevBuf oct_d, cyc_d, seed_d, nseed_d;
    JS_TRY(oct_d.alloc(M * 4, s));
    JS_TRY(cyc_d.alloc(M * 4, s));
    JS_TRY(seed_d.alloc((size_t)M * kSeedCap * 4, s));
    JS_TRY(nseed_d.alloc(M * 4, s));
    JS_CUDA(cudaMemsetAsync(nseed_d.p, 0, M * 4, s));
    c.seeds = seed_d.as<int32_t>();
    c.nseeds = nseed_d.as<int32_t>();
    std::vector<int32_t> ones(M, 1);
    JS_CUDA(cudaMemcpyAsync(oct_d.p, oct.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(cyc_d.p, ones.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaStreamSynchronize(s));
    std::unique_ptr<Dags> dg;
    JS_CUDA(cudaEventRecord(pe[0], s));
    if (d->opt.layering == JSWEEP_LAYERS_OCTANT) dg.reset(build_diagonals(d, s));
    JS_CUDA(cudaEventRecord(pe[1], s));
    c.lam = dg ? dg->level.as<int32_t>() : nullptr;
    c.oct = oct_d.as<int32_t>();
    c.cyc = cyc_d.as<int32_t>();
    if (dg) JS_CUDA(cudaMemsetAsync(c.cyc, 0, M * 4, s));
    {
        std::vector<float> d32(3 * M);
        for (int64_t i = 0; i < 3 * M; ++i) d32[i] = (float)d->quad->dirs[i];
        DevBuf dirs32;
        JS_TRY(dirs32.alloc(3 * M * 4, s));
        JS_CUDA(cudaMemcpyAsync(dirs32.p, d32.data(), 3 * M * 4, cudaMemcpyHostToDevice, s));
        const size_t shm = (size_t)M;
        if (shm > 48 * 1024)
            JS_CUDA(cudaFuncSetAttribute(k_classify, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        k_classify<<<(unsigned)((N + kClassifyThreads - 1) / kClassifyThreads), kClassifyThreads, shm, s>>>(
            c, dirs32.as<float>());
        JS_LAUNCH_CHECK();
        JS_CUDA(cudaStreamSynchronize(s));  // dirs32 is released on return
    }
    JS_CUDA(cudaEventRecord(pe[2], s));

    // ---- frontier loop with stall resolution
    const int B = d->opt.cycle_search_max;
    const int walk_max = 1 << 15;
    const size_t shmem = (size_t)kResolveWarps * (2 * B + (B + 3) / 4) * 4;
    JS_CUDA(cudaFuncSetAttribute(k_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmem));
    const int64_t max_steps = 4 * N + 1024;
    int32_t status[8] = {0, 0, 1, 0, 0, 0, 0, 0};
    int64_t step = 0;
    const int check_every = 16;
    int32_t last_remaining = -1;
    int no_progress_checks = 0;
    // peel: a grid of resident blocks over the step's frontier cells of every
    // direction (per-direction offsets in dynamic shared memory)
    // (kernels compiled for the mesh's face slots rounded up to 4, 6 or 7)
    const int fs = mesh->FS;
    void (*peel_k)(BuildCtx, int) = fs <= 4 ? k_peel<4> : fs <= 6 ? k_peel<6> : k_peel<7>;
    void (*walk_k)(BuildCtx, int, int, int) = fs <= 4 ? k_walk<4> : fs <= 6 ? k_walk<6> : k_walk<7>;
    const size_t off_shm = (size_t)(M + 1) * 8;
    if (off_shm > 48 * 1024)
        JS_CUDA(cudaFuncSetAttribute(peel_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)off_shm));
    int peel_per_sm = 0;
    JS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&peel_per_sm, peel_k, 256, off_shm));
    const int peel_blocks = device_sm_count() * std::max(1, peel_per_sm);
    // walks of a direction run in parallel over its candidates; a direction has
    // up to tens of thousands of them in a step on large meshes
    const int walk_blocks = (int)std::min<int64_t>(std::max<int64_t>(8, N / (256 * 16)), 64);
    // JSWEEP_BUILD_PROFILE=1: device time of each kernel of the frontier loop
    // (events around every launch; printed to stderr at the end of the build)
    const bool prof = std::getenv("JSWEEP_BUILD_PROFILE") != nullptr;
    std::vector<cudaEvent_t> pev;
    double kms[4] = {0, 0, 0, 0};
    auto prof_mark = [&](int k) {
        if (!prof) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        pev.push_back(e);
        (void)k;
    };
    // Cycles are searched for every kSearchEvery steps in the directions that
    // have stalled, and every kEagerEvery steps in every cyclic direction with
    // candidates (the candidates of the steps in between accumulate): the lags
    // found do not depend on when a component is found, only how long the cells
    // behind it wait.
    constexpr int kSearchEvery = 16, kEagerEvery = 16;
    static_assert(check_every % kEagerEvery == 0 && kEagerEvery % kSearchEvery == 0 && check_every % 2 == 0,
                  "a check period repeats the steps");
    const int Beager = d->eager_cap > 0 ? d->eager_cap : B;
    auto launch_step = [&](cudaStream_t st, int64_t stp, bool marks) {
        const int cur = (int)(stp & 1);
        const bool search = stp % kSearchEvery == kSearchEvery - 1;
        const int eager = stp % kEagerEvery == kEagerEvery - 1 ? 1 : 0;
        if (marks) prof_mark(0);
        peel_k<<<peel_blocks, 256, off_shm, st>>>(c, cur);
        if (marks) prof_mark(1);
        if (search) walk_k<<<dim3(walk_blocks, (unsigned)M), 256, 0, st>>>(c, cur ^ 1, eager, walk_max);
        if (marks) prof_mark(2);
        if (search) k_resolve<<<(unsigned)M, kResolveWarps * 32, shmem, st>>>(c, cur ^ 1, eager, B, Beager);
        if (marks) prof_mark(3);
        if (search) k_commit<<<64, 256, 0, st>>>(c, cur ^ 1);
        if (marks) prof_mark(4);
        return search ? 4 : 1;
    };
    // One check period (check_every steps) is captured once into a CUDA graph and
    // replayed: the steps of a period are the same launches every time (the
    // step parity and the search steps repeat), and the host then issues one
    // graph launch per period instead of a few launches per step.
    struct PeriodGraph {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;
        ~PeriodGraph() {
            if (exec) cudaGraphExecDestroy(exec);
            if (cap) cudaStreamDestroy(cap);
        }
    } period;
    int period_launches = 0;
    if (!prof && cudaStreamCreateWithFlags(&period.cap, cudaStreamNonBlocking) == cudaSuccess &&
        cudaStreamBeginCapture(period.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        for (int k = 0; k < check_every; ++k) period_launches += launch_step(period.cap, k, false);
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(period.cap, &g) == cudaSuccess && g) {
            if (cudaGraphInstantiate(&period.exec, g, 0) != cudaSuccess) period.exec = nullptr;
            cudaGraphDestroy(g);
        }
        cudaGetLastError();  // a failed capture falls back to launches step by step
    }
    // one status check: false to go on; true when done (rc = 0) or failed (rc)
    auto check_status = [&](int &rc) -> bool {
        rc = JSWEEP_OK;
        if (status[0] != 0) {
            if (status[0] == JSWEEP_ERR_CYCLE)
                set_error("dependency cycle in direction %d could not be broken within the search "
                          "cap of %d cells (raise jsweep_options.cycle_search_max)", status[1], B);
            else
                set_error("dag build: internal list capacity exceeded (status %d)", status[0]);
            rc = status[0];
            return true;
        }
        if (status[2] == 0) return true;
        // every step either processes cells or lags faces whose cells are
        // processed in the next one; a long run without progress is a bug
        no_progress_checks = status[2] == last_remaining ? no_progress_checks + 1 : 0;
        last_remaining = status[2];
        if (no_progress_checks > 16 || step > max_steps) {
            set_error("dag build did not finish after %lld steps", (long long)step);
            rc = JSWEEP_ERR_CYCLE;
            return true;
        }
        return false;
    };
    if (period.exec) {
        // Pipelined checks: period k + 1 is queued before period k's status is
        // read, so the device never waits for the host.  A period queued after
        // the last one needed finds every frontier empty and does nothing.
        struct HostStatus {
            cudaStream_t s = nullptr;
            int32_t *p = nullptr;
            cudaEvent_t ev[2] = {nullptr, nullptr};
            ~HostStatus() {
                if (s) cudaStreamSynchronize(s);  // a queued copy may still target p (early error return)
                if (p) cudaFreeHost(p);
                for (auto e : ev)
                    if (e) cudaEventDestroy(e);
            }
        } hs;
        hs.s = s;
        JS_CUDA(cudaMallocHost(&hs.p, 2 * 32));
        for (auto &e : hs.ev) JS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        int64_t launched = 0, checked = 0;
        auto launch_period = [&]() -> int {
            const int sl = (int)(launched & 1);
            JS_CUDA(cudaGraphLaunch(period.exec, s));
            note_launches(period_launches);
            JS_CUDA(cudaMemcpyAsync(hs.p + 8 * sl, c.status, 32, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaEventRecord(hs.ev[sl], s));
            ++launched;
            return JSWEEP_OK;
        };
        JS_TRY(launch_period());
        while (true) {
            JS_TRY(launch_period());
            const int sl = (int)(checked & 1);
            JS_CUDA(cudaEventSynchronize(hs.ev[sl]));
            ++checked;
            step = checked * check_every;
            std::memcpy(status, hs.p + 8 * sl, 32);
            int rc = JSWEEP_OK;
            if (check_status(rc)) {
                JS_CUDA(cudaStreamSynchronize(s));  // the period queued ahead
                if (rc != JSWEEP_OK) return rc;
                break;
            }
        }
    } else {
        while (true) {
            note_launches(launch_step(s, step, prof));
            if (prof && pev.size() >= 500) {  // fold the events of a few steps into the totals
                cudaStreamSynchronize(s);
                for (size_t i = 0; i + 4 < pev.size(); i += 5)
                    for (int k = 0; k < 4; ++k) {
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, pev[i + k], pev[i + k + 1]);
                        kms[k] += ms;
                    }
                for (auto e : pev) cudaEventDestroy(e);
                pev.clear();
            }
            JS_CUDA(cudaGetLastError());
            ++step;
            if (step % check_every == 0) {
                JS_CUDA(cudaMemcpyAsync(status, c.status, 32, cudaMemcpyDeviceToHost, s));
                JS_CUDA(cudaStreamSynchronize(s));
                int rc = JSWEEP_OK;
                if (check_status(rc)) {
                    if (rc != JSWEEP_OK) return rc;
                    break;
                }
            }
        }
    }

    if (prof) {
        cudaStreamSynchronize(s);
        for (size_t i = 0; i + 4 < pev.size(); i += 5)
            for (int k = 0; k < 4; ++k) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, pev[i + k], pev[i + k + 1]);
                kms[k] += ms;
            }
        for (auto e : pev) cudaEventDestroy(e);
        std::fprintf(stderr, "frontier loop: %lld steps; peel %.1f ms, walk %.1f ms, resolve %.1f ms, commit %.1f ms\n",
                     (long long)step, kms[0], kms[1], kms[2], kms[3]);
    }
    JS_CUDA(cudaEventRecord(pe[3], s));
    // ---- levels and masks back to [M][N]; the loop's state is released
    DevBuf msk;
    JS_TRY(d->level.alloc(MN * 4, s));
    JS_TRY(msk.alloc(MN * 4, s));
    k_ungroup<true><<<grid_for(SN / 8, 256, 152 * 16), 256, 0, s>>>(st_g.as<uint32_t>(), sdir_d.as<int32_t>(), N, S,
                                                                    d->level.as<uint32_t>());
    JS_LAUNCH_CHECK();
    k_ungroup<false><<<grid_for(SN / 8, 256, 152 * 16), 256, 0, s>>>(msk_g.as<uint32_t>(), sdir_d.as<int32_t>(), N,
                                                                     S, msk.as<uint32_t>());
    JS_LAUNCH_CHECK();
    const int32_t *lvl = d->level.as<int32_t>();
    c.msk = msk.as<uchar4>();
    JS_CUDA(cudaStreamSynchronize(s));  // the allocator may hand the released memory to another stream
    for (DevBuf *b : {&st_g, &msk_g, &stamp, &claim, &wclaim, &front, &cand}) b->release();
    // ---- levels per direction
    DevBuf lmax;
    JS_TRY(lmax.alloc(M * 4, s));
    JS_CUDA(cudaMemsetAsync(lmax.p, 0xff, M * 4, s));
    k_level_max<<<dim3(std::min<int64_t>(64, (N + 255) / 256), (unsigned)M), 256, 0, s>>>(lvl, N, M, lmax.as<int32_t>());
    JS_LAUNCH_CHECK();
    std::vector<int32_t> lm(M);
    JS_CUDA(cudaMemcpyAsync(lm.data(), lmax.p, M * 4, cudaMemcpyDeviceToHost, s));
    int32_t nlag_total = 0;
    JS_CUDA(cudaMemcpyAsync(&nlag_total, c.nlag, 4, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    d->nlevels.resize(M);
    d->lp_off.resize(M + 1);
    d->lp_off[0] = 0;
    d->Lmax = 0;
    for (int64_t m = 0; m < M; ++m) {
        d->nlevels[m] = (int64_t)lm[m] + 1;
        d->Lmax = std::max(d->Lmax, d->nlevels[m]);
        d->lp_off[m + 1] = d->lp_off[m] + d->nlevels[m] + 1;
    }
    if (d->Lmax >= (1ll << 24)) {
        set_error("too many levels (%lld)", (long long)d->Lmax);
        return JSWEEP_ERR_UNIMPLEMENTED;
    }

    // ---- level-major order (stable by cell id) and level_ptr
    int key_bits = 1;
    while ((1ll << key_bits) < d->Lmax) ++key_bits;
    DevBuf skeys;
    JS_TRY(d->order.alloc(MN * 4, s));
    JS_TRY(skeys.alloc(MN * 4, s));
    JS_TRY(radix_sort_segments(reinterpret_cast<const uint32_t *>(lvl), M, N, key_bits, nullptr,
                               d->order.as<int32_t>(), skeys.as<uint32_t>(), s));
    DevBuf lpoff_d, nlev_d;
    JS_TRY(d->lp.alloc(d->lp_off[M] * 4, s));
    JS_TRY(lpoff_d.alloc((M + 1) * 8, s));
    JS_TRY(nlev_d.alloc(M * 4, s));
    std::vector<int32_t> nl32(M);
    for (int64_t m = 0; m < M; ++m) nl32[m] = (int32_t)d->nlevels[m];
    JS_CUDA(cudaMemcpyAsync(lpoff_d.p, d->lp_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nlev_d.p, nl32.data(), M * 4, cudaMemcpyHostToDevice, s));
    k_level_ptr<<<dim3(std::min<int64_t>(64, (N + 255) / 256), (unsigned)M), 256, 0, s>>>(
        skeys.as<uint32_t>(), N, M, lpoff_d.as<int64_t>(), nlev_d.as<int32_t>(), d->lp.as<int32_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(d->mask.alloc(MN, s));
    k_mask_level_order<<<grid_for(MN, 256, 152 * 64), 256, 0, s>>>(c.msk, d->order.as<int32_t>(), N, M,
                                                                    d->mask.as<uint8_t>());
    JS_LAUNCH_CHECK();

    JS_CUDA(cudaEventRecord(pe[4], s));
    // ---- lag list sorted by (direction, face id)
    const int32_t T = std::min<int32_t>(nlag_total, (int32_t)lag_cap);
    d->T = T;
    JS_TRY(d->lag_ptr.alloc((M + 1) * 4, s));
    JS_TRY(d->lag_m.alloc(std::max<int64_t>(T, 1) * 4, s));
    JS_TRY(d->lag_face.alloc(std::max<int64_t>(T, 1) * 4, s));
    JS_TRY(d->lag_up.alloc(std::max<int64_t>(T, 1) * 4, s));
    JS_TRY(d->lag_dn.alloc(std::max<int64_t>(T, 1) * 4, s));
    if (T > 0) {
        DevBuf kf, km, km2, p1, p2;
        JS_TRY(kf.alloc(T * 4, s));
        JS_TRY(km.alloc(T * 4, s));
        JS_TRY(km2.alloc(T * 4, s));
        JS_TRY(p1.alloc(T * 4, s));
        JS_TRY(p2.alloc(T * 4, s));
        k_lag_keys<<<grid_for(T, 256), 256, 0, s>>>(c.lagall, T, kf.as<uint32_t>(), km.as<uint32_t>());
        JS_LAUNCH_CHECK();
        JS_TRY(radix_sort_segments(kf.as<uint32_t>(), 1, T, 31, nullptr, p1.as<int32_t>(), nullptr, s));
        k_gather_u32<<<grid_for(T, 256), 256, 0, s>>>(km.as<uint32_t>(), p1.as<int32_t>(), T, km2.as<uint32_t>());
        JS_LAUNCH_CHECK();
        int mbits = 1;
        while ((1ll << mbits) < M) ++mbits;
        JS_TRY(radix_sort_segments(km2.as<uint32_t>(), 1, T, mbits, p1.as<int32_t>(), p2.as<int32_t>(), nullptr, s));
        k_lag_scatter<<<grid_for(T, 256), 256, 0, s>>>(c.lagall, p2.as<int32_t>(), T, d->lag_m.as<int32_t>(),
                                                      d->lag_face.as<int32_t>(), d->lag_up.as<int32_t>(),
                                                      d->lag_dn.as<int32_t>());
        JS_LAUNCH_CHECK();
    }
    k_lag_ptr<<<grid_for(T + 1, 256), 256, 0, s>>>(d->lag_m.as<int32_t>(), T, M, d->lag_ptr.as<int32_t>());
    JS_LAUNCH_CHECK();
    std::vector<int32_t> lp32(M + 1);
    JS_CUDA(cudaMemcpyAsync(lp32.data(), d->lag_ptr.p, (M + 1) * 4, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    d->lag_ptr_h.assign(lp32.begin(), lp32.end());
    d->timing.build_steps = step;
    d->timing.build_stall_rounds = status[4];

    JS_CUDA(cudaEventRecord(pe[5], s));
    // ---- schedule layering
    d->layering = JSWEEP_LAYERS_LEVEL;
    d->s_order = d->order.as<int32_t>();
    d->s_mask = d->mask.as<uint8_t>();
    d->s_lp = d->lp.as<int32_t>();
    d->slayers = d->nlevels;
    d->sp_off = d->lp_off;
    d->Smax = d->Lmax;
    if (dg) {
        int rc = octant_layers(d, dg.get(), oct, c.msk, lpoff_d.as<int64_t>(), nlev_d.as<int32_t>(), s);
        if (rc != JSWEEP_OK) return rc;
    }
    JS_CUDA(cudaEventRecord(pe[6], s));
    JS_CUDA(cudaEventRecord(d->ev[1], s));
    JS_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, d->ev[0], d->ev[1]);
    d->timing.build_ms = ms;
    for (int i = 0; i < 6; ++i) {
        float t = 0.f;
        cudaEventElapsedTime(&t, pe[i], pe[i + 1]);
        d->timing.build_phase_ms[i] = t;
    }
    d->psi_lag.release();
    d->lag_R = 0;
    d->lag_prec = -1;
    return JSWEEP_OK;
}

}  // namespace js
