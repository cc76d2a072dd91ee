// Sweeps and source iteration of one problem on the device.
//
// Work unit: up to `cluster_cells` (<= 32 / SPLIT) consecutive cells of one
// schedule layer of one direction (vertex clustering, Sec. V-C); one warp
// processes a unit, SPLIT lanes per cell.  Cells of one layer never depend on
// each other, so a unit needs no internal ordering.
//
// Two schedules (Sec. V-B patch-angle parallelism: all directions progress
// together):
//   level-synchronous: one launch per schedule slot covering that slot's
//     layers of all directions; the launches are captured once into a CUDA
//     graph and replayed, each slot starting early (programmatic dependent
//     launch) and waiting only before its upwind reads.  By default the slot
//     kernel (k_sweep_level_coef) reads each cell-direction's face
//     coefficients (Omega.A per face slot and the upwind ids) from a stream
//     laid out in sweep order (k_coef_fill, once per handle); k_sweep_level
//     computes them from the cell geometry instead (no_face_stream).  With
//     tail_units, the last small slots run in one launch of one block per
//     direction (k_sweep_tail), layer after layer.
//   data-driven (persistent): one launch of resident warps; unit t of the
//     slot-ordered table goes to warp t mod W, and each cell waits (bounded
//     spin, acquire) for its own upwind cells' epoch flags, then releases its
//     own.  The table is a topological order of every direction's graph, so
//     the smallest unfinished unit always has its producers done: no
//     deadlock while every warp is resident.
//
// Per-cell solve (step scheme, Sec. II-C): see solve_cell in sweep_cell.cuh.
//
// Layouts: psi [N][M][R] (cell-major: a cell's directions are contiguous, the
// R right-hand sides of one cell-direction form one 16/32-byte piece), source
// records [N][RS] (S V of each rhs, then sigma_t V), lagged values [T][R],
// face-coefficient records [M][N] in sweep order (coef_record_bytes each).
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "sweep_cell.cuh"

namespace js {

using namespace dev;

namespace {

// Level-synchronous sweep: one launch per time slot; a warp handles one unit
// of 32 / SPLIT cells.
template <class T, int R, int SPLIT, int MAXF>
__global__ void __launch_bounds__(kLevelWarps * 32) k_sweep_level(SweepArgs<T> a, int64_t u0, int64_t nu) {
    pdl_launch_next();
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
    if (t >= nu) return;
    const int4 u = a.units[u0 + t];
    const int cell = lane / SPLIT, sub = lane % SPLIT;
    if (cell < u.z && JS_IN_RANGE(a, u.x, a.M, 5) && JS_IN_RANGE(a, (int64_t)u.y + cell, a.N, 4)) {
        const int64_t idx = (int64_t)u.x * a.N + u.y + cell;
        solve_cell<T, R, SPLIT, MAXF, false, true>(a, u.x, __ldg(a.order + idx), __ldg(a.mask + idx), sub, nullptr,
                                                   0, nullptr, 0);
    }
}

// Level-synchronous sweep reading the precomputed face coefficients (SEQ: the
// records hold upwind positions and psi has a sweep-order copy, see
// solve_cell_coef).
// The kernel is bound by how many warps have memory requests in flight: it
// is compiled for 48 resident warps per SM (40 registers), which measured
// faster than 40 (48 registers) or 64 (32 registers, with spills).
template <class T, int R, int SPLIT, int MAXF, bool SEQ, bool MG>
__global__ void __launch_bounds__(kLevelWarps * 32, 48 / kLevelWarps)
    k_sweep_level_coef(SweepArgs<T> a, int64_t u0, int64_t nu, const unsigned char *coef) {
    pdl_launch_next();
    constexpr int RB = coef_record_bytes<T, MAXF>();
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * kLevelWarps + (threadIdx.x >> 5);
    if (t >= nu) return;
    const uint64_t pol_stream = l2_evict_first();
    const int4 u = ldg_hint(a.units + u0 + t, pol_stream);
    const int cell = lane / SPLIT, sub = lane % SPLIT;
    if (cell < u.z && JS_IN_RANGE(a, u.x, a.M, 5) && JS_IN_RANGE(a, (int64_t)u.y + cell, a.N, 4)) {
        const int64_t idx = (int64_t)u.x * a.N + u.y + cell;
        solve_cell_coef<T, R, SPLIT, MAXF, SEQ, MG>(a, u.x, ldg_hint(a.order + idx, pol_stream),
                                                ldg_hint(a.mask + idx, pol_stream), sub, coef + idx * RB, pol_stream,
                                                [] {
                                                    pdl_wait_prev();  // upwind values come from earlier slots
                                                    return true;
                                                },
                                                idx);
    }
}

// The tail of a level-synchronous sweep, one block per direction: the last
// slots, each too small to fill the GPU, are swept by block m for direction m,
// layer after layer with a block barrier between layers, instead of by one
// launch per slot.  A layer depends only on earlier layers of its own
// direction (the per-direction dependency graph), so the blocks never wait for
// one another; the layers before first_layer were swept by the slot launches
// that precede this one.
template <class T, int R, int SPLIT, int MAXF, bool SEQ, bool MG>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_sweep_tail(SweepArgs<T> a, const int32_t *lp, const int64_t *lp_off, const int32_t *nlev, int first_layer,
                 const unsigned char *coef) {
    constexpr int RB = coef_record_bytes<T, MAXF>();
    constexpr int per_pass = kWarpsPerBlock * 32 / SPLIT;  // cells of a layer solved at once
    const int m = blockIdx.x;
    const int cell = threadIdx.x / SPLIT, sub = threadIdx.x % SPLIT;
    const uint64_t pol_stream = l2_evict_first();
    const int L = nlev[m];
    const int32_t *lpm = lp + lp_off[m];
    pdl_wait_prev();  // the slot launches before the tail are complete
    for (int l = first_layer; l < L; ++l) {
        const int p1 = lpm[l + 1];
        for (int p = lpm[l] + cell; p < p1; p += per_pass) {
            if (!JS_IN_RANGE(a, p, a.N, 4)) continue;
            const int64_t idx = (int64_t)m * a.N + p;
            solve_cell_coef<T, R, SPLIT, MAXF, SEQ, MG>(a, m, ldg_hint(a.order + idx, pol_stream),
                                                    ldg_hint(a.mask + idx, pol_stream), sub, coef + idx * RB,
                                                    pol_stream, [] { return true; }, idx);
        }
        __syncthreads();  // this layer's psi is stored before the next layer reads it
    }
}

// Position of every cell in each direction's sweep order: pos[m][order[m][p]] = p.
__global__ void k_sweep_positions(const int32_t *order, int64_t N, int64_t M, int32_t *pos) {
    const int64_t total = N * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N;
        pos[m * N + order[i]] = (int32_t)(i - m * N);
    }
}

// Face-coefficient records of every (direction, position) of the sweep order.
// With pos (not null) an interior neighbour is recorded as its position in the
// direction's sweep order instead of its cell id.
template <class T, int MAXF>
__global__ void k_coef_fill(const int32_t *order, const typename V4<T>::type *geo, const T *dirs, int64_t N,
                            int64_t M, int FS, int GS, const int32_t *pos, unsigned char *coef) {
    constexpr int RB = coef_record_bytes<T, MAXF>();
    const int64_t total = N * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N;
        const int32_t c = order[i];
        const T ox = dirs[4 * m], oy = dirs[4 * m + 1], oz = dirs[4 * m + 2];
        alignas(16) unsigned char rec[RB];
        T dk[MAXF];
        int32_t nbk[MAXF];
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            if (k < FS) {
                const typename V4<T>::type g = geo[(int64_t)c * GS + k];
                dk[k] = face_dot(ox, oy, oz, g.x, g.y, g.z);
                nbk[k] = nbr_bits<T>(g);
                if (pos && nbk[k] >= 0) nbk[k] = pos[m * N + nbk[k]];
            } else {
                dk[k] = T(0);
                nbk[k] = INT32_MIN;
            }
        }
        memset(rec, 0, RB);
        memcpy(rec, dk, MAXF * sizeof(T));
        memcpy(rec + MAXF * sizeof(T), nbk, MAXF * 4);
        float4 *dst = reinterpret_cast<float4 *>(coef + i * RB);
#pragma unroll
        for (int w = 0; w < RB / 16; ++w) {
            float4 v;
            memcpy(&v, rec + 16 * w, 16);
            dst[w] = v;
        }
    }
}

// Data-driven sweep (Listing 1's readiness, per cell): units are taken in
// schedule order, unit t by resident warp t mod W; each cell waits only for
// its own upwind cells' flags, then publishes its psi and its flag with
// release ordering.  The schedule is a topological order of every
// direction's graph, so the smallest unfinished unit always has its producers
// done and its warp free: the sweep cannot deadlock while all W warps are
// resident (the grid is sized from the occupancy calculator).
template <class T, int R, int SPLIT, int MAXF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_sweep_dd(SweepArgs<T> a, int64_t n_units, int *flags, int epoch, int want, int *err, long long timeout) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * kWarpsPerBlock;
    const int cell = lane / SPLIT, sub = lane % SPLIT;
    for (int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); t < n_units; t += W) {
        if (__shfl_sync(0xffffffffu, lane == 0 ? ld_volatile(err) : 0, 0) != 0) return;
        const int4 u = a.units[t];
        bool ok = true;
        int c = -1;
        if (cell < u.z && JS_IN_RANGE(a, u.x, a.M, 5) && JS_IN_RANGE(a, (int64_t)u.y + cell, a.N, 4)) {
            const int64_t idx = (int64_t)u.x * a.N + u.y + cell;
            c = __ldg(a.order + idx);
            if (JS_IN_RANGE(a, c, a.N, 1))
                ok = solve_cell<T, R, SPLIT, MAXF, true>(a, u.x, c, __ldg(a.mask + idx), sub, flags, want, err,
                                                         timeout);
            else
                c = -1;  // bounds-checked builds: a bad cell id is neither solved nor released
        }
        if constexpr (SPLIT == 1) {
            if (c >= 0 && ok) st_release(flags + (int64_t)c * a.M + u.x, epoch);
        } else {
            // the lanes of a cell publish together: each makes its own stores
            // visible, then the first lane of the cell releases the flag
            __threadfence();
            __syncwarp();
            if (c >= 0 && ok && sub == 0) st_release(flags + (int64_t)c * a.M + u.x, epoch);
        }
        if (__any_sync(0xffffffffu, !ok)) return;
    }
}

// Data-driven persistent sweep with ready queues and dependency counters
// (Listing 1: the counts, the queue Q and its dequeue; vertex clustering,
// Sec. V-C; priority, Sec. V-D).  The work units (up to 32 / SPLIT cells of
// one layer of one direction) of direction m sit in the table in depth order
// (layer by layer, dir_ptr[m] .. dir_ptr[m+1]); cursor[m] is m's queue head
// and done[m] counts m's finished units.  A warp dequeues one unit of its
// direction (one atomic on m's own cursor; every direction's cursor and
// counter have a 128-byte line to themselves, since same-address atomics
// serialise); a unit of layer l needs every unit of m's layers before l (its
// wait target u.w), so its cells wait (bounded, acquire) until done[m] reaches
// it, then read their upwind values, solve and store, and the warp adds one
// to done[m] after a fence.  Warps start on direction (warp mod M) and move to
// the next direction when theirs has no units left; they return when a whole
// round of directions had none.  Within a direction units are dequeued in
// order and wait only for earlier units, so the first unfinished unit of a
// direction is either running or not yet dequeued by anyone: some warp can
// always progress, whether or not every block is resident.  The face records
// hold upwind positions and psi has its sweep-order copy (solve_cell_coef,
// SEQ).
constexpr int kQueueStride = 32;  // ints between two directions' cursors / counters (128 bytes)

template <class T, int R, int SPLIT, int MAXF, bool MG>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, 6)
    k_sweep_queue(SweepArgs<T> a, const int64_t *dir_ptr, const unsigned char *coef, unsigned *cursor, int *done,
                  int extra, int *err, long long timeout) {
    constexpr int RB = coef_record_bytes<T, MAXF>();
    const int lane = threadIdx.x & 31;
    const int cell = lane / SPLIT, sub = lane % SPLIT;
    const uint64_t pol = l2_evict_first();
    int m = (int)(((int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5)) % a.M);
    int empty = 0;  // directions in a row found without units
    while (empty < a.M) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(cursor + (int64_t)m * kQueueStride, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        const int64_t u0 = dir_ptr[m], nm = dir_ptr[m + 1] - u0;
        if ((int64_t)t >= nm) {
            m = m + 1 == a.M ? 0 : m + 1;
            ++empty;
            continue;
        }
        empty = 0;
        const int4 u = ldg_hint(a.units + u0 + t, pol);
        int *dm = done + (int64_t)m * kQueueStride;
        bool ok = true;
        if (cell < u.z && JS_IN_RANGE(a, u.x, a.M, 5) && JS_IN_RANGE(a, (int64_t)u.y + cell, a.N, 4)) {
            const int64_t idx = (int64_t)u.x * a.N + u.y + cell;
            const int want = u.w + extra;
            ok = solve_cell_coef<T, R, SPLIT, MAXF, true, MG>(
                a, u.x, ldg_hint(a.order + idx, pol), ldg_hint(a.mask + idx, pol), sub, coef + idx * RB, pol,
                [&] {
                    if (ld_acquire(dm) >= want) return true;
                    const long long t0 = clock64();
                    int ns = 32;
                    while (ld_acquire(dm) < want) {
                        if (ld_volatile(err) != 0) return false;
                        if (clock64() - t0 > timeout) {
                            atomicCAS(err, 0, 1);
                            return false;
                        }
                        __nanosleep(ns);
                        ns = ns < 256 ? 2 * ns : 256;
                    }
                    return true;
                },
                idx);
        }
        // the warp's stores are visible device-wide before its unit counts as done
        __threadfence();
        if (__any_sync(0xffffffffu, !ok)) return;
        if (lane == 0) atomicAdd(dm, 1);
    }
}

// ---- unit schedule ------------------------------------------------------------------
__global__ void k_unit_counts(const int32_t *lp, const int64_t *lp_off, const int32_t *nlev, int64_t M,
                              int64_t Lmax, int U, int64_t *ucnt) {
    const int64_t total = M * Lmax;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = i / Lmax, l = i - m * Lmax;
        int64_t n = 0;
        if (l < nlev[m]) n = lp[lp_off[m] + l + 1] - lp[lp_off[m] + l];
        ucnt[i] = (n + U - 1) / U;
    }
}

// Per-slot unit counts, laid out per slot in grouped direction order (qpos[m]).
__global__ void k_unit_slots(const int64_t *ucnt, const int32_t *off, const int32_t *qpos, int64_t M, int64_t Lmax,
                             int64_t Tmax, int64_t *cnt2) {
    const int64_t total = M * Lmax;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m = i / Lmax, l = i - m * Lmax;
        int64_t t = l + off[m];
        if (t < Tmax) cnt2[t * M + qpos[m]] = ucnt[i];
    }
}

// Fills the unit table.  Inside a slot t the directions are laid out in grouped
// order (octant by octant: gmem, group g = [gstart[g], gstart[g+1]), qpos[m] =
// position of m).  Either direction by direction (interleave = 0), or with the
// units of a group interleaved: chunk 0 of each of its directions, chunk 1 of
// each, ... (interleave = 1), so that chunks covering nearby cells for
// different directions sit next to each other.
__global__ void k_unit_fill(const int32_t *lp, const int64_t *lp_off, const int32_t *nlev, const int64_t *ucnt,
                            const int64_t *wscan, const int64_t *base2, const int64_t *cnt2, const int32_t *off,
                            int64_t M, int64_t Lmax, int U, const int32_t *gmem, const int32_t *gstart,
                            const int32_t *gof, const int32_t *qpos, int interleave, int4 *units) {
    // one warp per (direction, layer), lanes over its units
    const int64_t total = M * Lmax;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < total; i += warps) {
        int64_t m = i / Lmax, l = i - m * Lmax;
        if (l >= nlev[m]) continue;
        int32_t p0 = lp[lp_off[m] + l], p1 = lp[lp_off[m] + l + 1];
        int64_t nu = ucnt[i];
        const int64_t t = l + off[m];
        int32_t wait = (int32_t)(wscan[i] - wscan[m * Lmax]);
        if (!interleave) {
            const int64_t b = base2[t * M + qpos[m]];
            for (int64_t j = lane; j < nu; j += 32) {
                int32_t s = p0 + (int32_t)(j * U);
                units[b + j] = make_int4((int)m, s, min(U, p1 - s), wait);
            }
            continue;
        }
        const int g = gof[m];
        const int64_t gb = base2[t * M + gstart[g]];
        for (int64_t j = lane; j < nu; j += 32) {
            int64_t pos = gb;
            for (int q = gstart[g]; q < gstart[g + 1]; ++q) {
                const int64_t uq = cnt2[t * M + q];
                pos += uq < j ? uq : j;                 // chunks 0..j-1 of every direction of the group
                if (gmem[q] < m && uq > j) pos += 1;    // chunk j of the group's directions before m
            }
            int32_t s = p0 + (int32_t)(j * U);
            units[pos] = make_int4((int)m, s, min(U, p1 - s), wait);
        }
    }
}

// Direction-major unit table: the units of (m, l) start at wscan[m * Lmax + l]
// (the exclusive scan of the unit counts in direction-then-layer order), and
// each waits for the units of m's layers before l.
__global__ void k_unit_fill_dir(const int32_t *lp, const int64_t *lp_off, const int32_t *nlev, const int64_t *ucnt,
                                const int64_t *wscan, int64_t M, int64_t Lmax, int U, int4 *units) {
    // one warp per (direction, layer), lanes over its units
    const int64_t total = M * Lmax;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < total; i += warps) {
        const int64_t m = i / Lmax, l = i - m * Lmax;
        if (l >= nlev[m]) continue;
        const int32_t p0 = lp[lp_off[m] + l], p1 = lp[lp_off[m] + l + 1];
        const int32_t wait = (int32_t)(wscan[i] - wscan[m * Lmax]);
        for (int64_t j = lane; j < ucnt[i]; j += 32) {
            const int32_t s = p0 + (int32_t)(j * U);
            units[wscan[i] + j] = make_int4((int)m, s, min(U, p1 - s), wait);
        }
    }
}

// ---- patch tasks ------------------------------------------------------------------------
inline bool patch_prio(int p) { return p == JSWEEP_PRIO_PATCH || p == JSWEEP_PRIO_PATCH_SLBD; }

// Triple i = (direction m, patch s, layer l), task-major: i = tri_off[m] + s * L_m + l.
__device__ __forceinline__ void patch_triple(int64_t i, const int64_t *tri_off, int64_t M, const int32_t *nlev,
                                             int64_t &m, int &s, int &l) {
    int64_t lo = 0, hi = M;  // largest m with tri_off[m] <= i
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (tri_off[mid] <= i) lo = mid;
        else hi = mid;
    }
    m = lo;
    const int64_t r = i - tri_off[m];
    const int L = nlev[m];
    s = (int)(r / L);
    l = (int)(r - (int64_t)s * L);
}

__device__ __forceinline__ int lower_bound_id(const int32_t *row, int lo, int hi, int32_t key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (row[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Cells of layer l of direction m that lie in patch s: [a, b) in the layer-major
// order (a layer's cells are sorted by id, and a patch is an id range).
__device__ __forceinline__ void patch_run(const int32_t *order, const int32_t *lp, const int64_t *lp_off, int64_t N,
                                          int nslab, int64_t m, int s, int l, int &a, int &b) {
    const int32_t *row = order + m * N;
    const int pa = lp[lp_off[m] + l], pb = lp[lp_off[m] + l + 1];
    const int32_t lo_id = (int32_t)((int64_t)s * N / nslab), hi_id = (int32_t)((int64_t)(s + 1) * N / nslab);
    a = lower_bound_id(row, pa, pb, lo_id);
    b = lower_bound_id(row, a, pb, hi_id);
}

__global__ void k_patch_counts(const int32_t *order, const int32_t *lp, const int64_t *lp_off, const int32_t *nlev,
                               const int64_t *tri_off, int64_t M, int64_t N, int nslab, int U, int64_t total,
                               int64_t *cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m;
        int s, l, a, b;
        patch_triple(i, tri_off, M, nlev, m, s, l);
        patch_run(order, lp, lp_off, N, nslab, m, s, l, a, b);
        cnt[i] = (b - a + U - 1) / U;
    }
}

__global__ void k_patch_task_max(const int64_t *uoff, const int64_t *cnt, const int64_t *tri_off, const int32_t *nlev,
                                 int64_t M, int nslab, unsigned long long *maxk) {
    const int64_t tasks = M * nslab;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tasks; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = t / nslab, s = t - m * nslab;
        const int64_t first = tri_off[m] + s * nlev[m], last = first + nlev[m] - 1;
        atomicMax(maxk, (unsigned long long)(uoff[last] + cnt[last] - uoff[first]));
    }
}

// Unit k of task (m, s) goes to table position task + W * k, so that the
// data-driven kernel (unit t on warp t mod W) gives each task to one warp,
// which runs the task's units in layer order.
__global__ void k_patch_fill(const int32_t *order, const int32_t *lp, const int64_t *lp_off, const int32_t *nlev,
                             const int64_t *tri_off, int64_t M, int64_t N, int nslab, int U, int64_t total,
                             const int64_t *uoff, int64_t W, int4 *units) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m;
        int s, l, a, b;
        patch_triple(i, tri_off, M, nlev, m, s, l);
        patch_run(order, lp, lp_off, N, nslab, m, s, l, a, b);
        const int64_t task = m * nslab + s;
        const int64_t k0 = uoff[i] - uoff[tri_off[m] + (int64_t)s * nlev[m]];
        for (int j = 0; a + j * U < b; ++j)
            units[task + W * (k0 + j)] = make_int4((int)m, a + j * U, min(U, b - a - j * U), 0);
    }
}

// ---- SLBD order of patch tasks (Sec. V-D) ----------------------------------------------
// Patch of cell c: the largest s with floor(s N / nslab) <= c (patches are id ranges).
__device__ __forceinline__ int patch_of(int64_t c, int64_t N, int nslab) {
    int s = (int)(c * nslab / N);
    while (s + 1 < nslab && (int64_t)(s + 1) * N / nslab <= c) ++s;
    while (s > 0 && (int64_t)s * N / nslab > c) --s;
    return s;
}

// Local boundary distance, breadth first: 0 for a cell with a face neighbour
// in another patch, else 1 + the smallest distance among its neighbours; -1
// until reached (a patch without another patch beside it keeps -1).
__global__ void k_bdist_init(const int32_t *nbr, int FS, int64_t N, int nslab, int32_t *dist) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int ps = patch_of(c, N, nslab);
        int32_t d = -1;
        for (int k = 0; k < FS; ++k) {
            const int32_t nb = nbr[c * FS + k];
            if (nb >= 0 && patch_of(nb, N, nslab) != ps) d = 0;
        }
        dist[c] = d;
    }
}

// One breadth-first round: cells not yet reached that touch a cell at distance
// r get r + 1 (writes of r + 1 do not disturb the reads of r).
__global__ void k_bdist_step(const int32_t *nbr, int FS, int64_t N, int32_t r, int32_t *dist, int *changed) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        if (dist[c] >= 0) continue;
        bool hit = false;
        for (int k = 0; k < FS; ++k) {
            const int32_t nb = nbr[c * FS + k];
            if (nb >= 0 && dist[nb] == r) hit = true;
        }
        if (hit) {
            dist[c] = r + 1;
            *changed = 1;
        }
    }
}

// Units of every (direction, patch, layer) run in id order, densely (unit j of
// triple i at uoff[i] + j), each with the sort key (i << 8) | the smallest
// local boundary distance of its cells (unreached: 255).
__global__ void k_patch_dense(const int32_t *order, const int32_t *lp, const int64_t *lp_off, const int32_t *nlev,
                              const int64_t *tri_off, int64_t M, int64_t N, int nslab, int U, int64_t total,
                              const int64_t *uoff, const int32_t *dist, int4 *du, uint32_t *dkey) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t m;
        int s, l, a, b;
        patch_triple(i, tri_off, M, nlev, m, s, l);
        patch_run(order, lp, lp_off, N, nslab, m, s, l, a, b);
        for (int j = 0; a + j * U < b; ++j) {
            const int p0 = a + j * U, z = min(U, b - p0);
            int key = 255;
            for (int q = 0; q < z; ++q) {
                const int32_t dv = dist[order[m * N + p0 + q]];
                if (dv >= 0) key = min(key, min(dv, 254));
            }
            du[uoff[i] + j] = make_int4((int)m, p0, z, 0);
            dkey[uoff[i] + j] = ((uint32_t)i << 8) | (uint32_t)key;
        }
    }
}

// The dense units in key order (a stable sort: within a run, by distance,
// then id) into the task table: the q-th sorted unit is the (q - uoff[i])-th of
// its run i.
__global__ void k_patch_scatter(const int4 *du, const uint32_t *dkey, const int32_t *perm, int64_t n,
                                const int64_t *uoff, const int64_t *tri_off, const int32_t *nlev, int64_t M,
                                int nslab, int64_t W, int4 *units) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = perm[q];
        const int64_t i = dkey[e] >> 8;
        int64_t m;
        int s, l;
        patch_triple(i, tri_off, M, nlev, m, s, l);
        const int64_t task = m * nslab + s;
        const int64_t k0 = uoff[i] - uoff[tri_off[m] + (int64_t)s * nlev[m]];
        units[task + W * (k0 + (q - uoff[i]))] = du[e];
    }
}

// ---- emission, phi, residual, lag update ----------------------------------------------
template <class T, int R>
__global__ void k_emission(const T *sig, const T *cr, const T *q, const T *phi, const T *vol, int64_t N,
                           int nrhs, T *srcv) {
    constexpr int RS = src_stride<R>();
    const T four_pi = T(4.0 * 3.141592653589793);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        T V = vol[c], s = sig[c];
        T cs = cr ? cr[c] * s : T(0);
        T out[RS];
#pragma unroll
        for (int r = 0; r < RS; ++r) out[r] = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < nrhs) {
                T p = phi ? phi[(int64_t)r * N + c] : T(0);
                out[r] = (fma_rn(cs, p, q[(int64_t)r * N + c]) / four_pi) * V;  // as k_emission_batch
            }
        }
        out[R] = s * V;
#pragma unroll
        for (int r = 0; r < RS; ++r) srcv[c * RS + r] = out[r];
    }
}

// Multigroup scattering source (the multigroup transport equation of the
// appendix, Alg. 1 step 2.1): every group's angular source from the previous
// iterate of all groups, S_g = (sum_h sigma_s[h][g] phi_h + q_g) / (4 pi),
// h in increasing order.  sigma_s [G][G][N] ([h][g]: rate from group h into
// group g), q and src [G][N], phi [G][N] or null (phi = 0).
template <class T>
__global__ void k_emission_mg(const T *sigma_s, const T *q, const T *phi, int64_t N, int G, T *src) {
    const T four_pi = T(4.0 * 3.141592653589793);
    const int64_t total = (int64_t)G * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i / N, c = i - g * N;
        T sum = T(0);
        if (phi)
            for (int h = 0; h < G; ++h) sum = fma_rn(sigma_s[((int64_t)h * G + g) * N + c], phi[(int64_t)h * N + c], sum);
        src[i] = add_rn(sum, q[i]) / four_pi;
    }
}

// Angular source given directly: records of S V and sigma_t V.
template <class T, int R>
__global__ void k_source_prep(const T *sig, const T *src, const T *vol, int64_t N, int nrhs, T *srcv) {
    constexpr int RS = src_stride<R>();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        T V = vol[c];
        T out[RS];
#pragma unroll
        for (int r = 0; r < RS; ++r) out[r] = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) out[r] = r < nrhs ? src[(int64_t)r * N + c] * V : T(0);
        out[R] = sig[c] * V;
#pragma unroll
        for (int r = 0; r < RS; ++r) srcv[c * RS + r] = out[r];
    }
}

// Source records of G groups riding the right-hand-side dimension: S_g V at
// [g], sigma_t,g V at [R + g] (src and sig [G][N]; the same products as
// k_source_prep of each group alone).
template <class T, int R>
__global__ void k_source_prep_mg(const T *sig, const T *src, const T *vol, int64_t N, int G, T *srcv) {
    constexpr int RS = src_stride<R>();
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const T V = vol[c];
        T out[RS];
#pragma unroll
        for (int r = 0; r < RS; ++r) out[r] = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < G) {
                out[r] = src[(int64_t)r * N + c] * V;
                out[R + r] = sig[(int64_t)r * N + c] * V;
            }
        }
#pragma unroll
        for (int r = 0; r < RS; ++r) srcv[c * RS + r] = out[r];
    }
}

template <class T, int R>
__global__ void k_phi(const T *psi, const T *w, int64_t N, int M, int nrhs, T *phi) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < N; c += warps) {
        T v[R];
        phi_warp<T, R>(psi + (int64_t)c * M * R, w, M, lane, v);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (lane == 0 && r < nrhs) phi[(int64_t)r * N + c] = v[r];
    }
}

template <class T, int R>
__global__ void k_lag_update(const T *psi, const int32_t *lag_m, const int32_t *lag_up, int64_t Tl, int64_t M,
                             T *psi_lag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < Tl; j += (int64_t)gridDim.x * blockDim.x) {
        T v[R];
        load_cg<T, R>(psi + ((int64_t)lag_up[j] * M + lag_m[j]) * R, v);
#pragma unroll
        for (int r = 0; r < R; ++r) psi_lag[j * R + r] = v[r];
    }
}

// FP64 residual accumulators: acc[2r] = max |phi_new - phi_old|, acc[2r+1] = max |phi_new|
// (non-negative doubles compare like their bit patterns).
template <class T>
__global__ void k_resid(const T *pn, const T *po, int64_t N, unsigned long long *acc) {
    const int r = blockIdx.y;
    double dmax = 0.0, pmax = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        double a = (double)pn[(int64_t)r * N + c];
        double b = po ? (double)po[(int64_t)r * N + c] : 0.0;
        dmax = fmax(dmax, fabs(a - b));
        pmax = fmax(pmax, fabs(a));
    }
    for (int off = 16; off > 0; off >>= 1) {
        dmax = fmax(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
        pmax = fmax(pmax, __shfl_down_sync(0xffffffffu, pmax, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(acc + 2 * r, (unsigned long long)__double_as_longlong(dmax));
        atomicMax(acc + 2 * r + 1, (unsigned long long)__double_as_longlong(pmax));
    }
}

__global__ void k_resid_final(const unsigned long long *acc, int nrhs, double *resid) {
    if (threadIdx.x != 0) return;
    double worst = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        double d = __longlong_as_double((long long)acc[2 * r]);
        double p = __longlong_as_double((long long)acc[2 * r + 1]);
        double v = p > 0.0 ? d / p : (d > 0.0 ? INFINITY : 0.0);
        resid[r] = v;
        worst = fmax(worst, v);
    }
    resid[nrhs] = worst;
}

template <class T, int R>
__global__ void k_psi_out(const T *psi, int64_t N, int M, int nrhs, T *out) {
    const int64_t total = (int64_t)M * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i / M, m = i - c * M;  // i = c * M + m (psi order)
        T v[R];
        load_cg<T, R>(psi + i * R, v);
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r < nrhs) out[((int64_t)r * M + m) * N + c] = v[r];
    }
}

int pad_rhs(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8; }

}  // namespace

// ---- unit tables ------------------------------------------------------------------------
// Patch-task table (JSWEEP_PRIO_PATCH, JSWEEP_PRIO_PATCH_SLBD): patches are id
// ranges; as many as resident warps allow (directions x patches <=
// resident_warps).  With SLBD the units of every (task, layer) run are
// ordered by their cells' local boundary distance (Sec. V-D), provided the
// runs can be numbered in 24 bits (else they keep id order).
static int ensure_units_patch(Dags *d, int U, int64_t resident_warps, cudaStream_t s, int prio) {
    const int64_t M = d->M, N = d->N;
    if (resident_warps < M) {
        set_error("patch tasks need at least one resident warp per direction (%lld directions, %lld warps)",
                  (long long)M, (long long)resident_warps);
        return JSWEEP_ERR_UNIMPLEMENTED;
    }
    const int nslab = (int)std::min<int64_t>(resident_warps / M, N);
    const int64_t tasks = M * nslab;
    const int64_t W = (tasks + kWarpsPerBlock - 1) / kWarpsPerBlock * kWarpsPerBlock;
    UnitTable &ut = d->ut;
    if (ut.mode == JSWEEP_MODE_PERSISTENT && ut.priority == prio && ut.cluster == U && ut.warps == W)
        return JSWEEP_OK;
    std::vector<int64_t> tri(M + 1, 0);
    std::vector<int32_t> nl32(M);
    for (int64_t m = 0; m < M; ++m) {
        nl32[m] = (int32_t)d->slayers[m];
        tri[m + 1] = tri[m] + (int64_t)nslab * d->slayers[m];
    }
    const int64_t total = tri[M];
    DevBuf tri_d, nlev_d, lpoff_d, cnt, uoff, maxk;
    JS_TRY(tri_d.alloc((M + 1) * 8, s));
    JS_TRY(nlev_d.alloc(M * 4, s));
    JS_TRY(lpoff_d.alloc((M + 1) * 8, s));
    JS_TRY(cnt.alloc(total * 8, s));
    JS_TRY(uoff.alloc(total * 8, s));
    JS_TRY(maxk.alloc(8, s));
    JS_CUDA(cudaMemcpyAsync(tri_d.p, tri.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nlev_d.p, nl32.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(lpoff_d.p, d->sp_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemsetAsync(maxk.p, 0, 8, s));
    k_patch_counts<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(d->s_order, d->s_lp, lpoff_d.as<int64_t>(),
                                                                  nlev_d.as<int32_t>(), tri_d.as<int64_t>(), M, N,
                                                                  nslab, U, total, cnt.as<int64_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(scan_exclusive_i64(cnt.as<int64_t>(), uoff.as<int64_t>(), total, s));
    k_patch_task_max<<<grid_for(tasks, 256, 4096), 256, 0, s>>>(uoff.as<int64_t>(), cnt.as<int64_t>(),
                                                                tri_d.as<int64_t>(), nlev_d.as<int32_t>(), M, nslab,
                                                                reinterpret_cast<unsigned long long *>(maxk.p));
    JS_LAUNCH_CHECK();
    unsigned long long kmax = 0;
    JS_CUDA(cudaMemcpyAsync(&kmax, maxk.p, 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    const int64_t n_units = W * (int64_t)kmax;
    JS_TRY(ut.units.alloc((size_t)std::max<int64_t>(n_units, 1) * 16, s));
    JS_CUDA(cudaMemsetAsync(ut.units.p, 0, (size_t)std::max<int64_t>(n_units, 1) * 16, s));  // empty units pad
    if (prio == JSWEEP_PRIO_PATCH_SLBD && total < (1ll << 24)) {
        // local boundary distances, then the runs' units sorted by (run, distance)
        const int FS = d->mesh->FS;
        const int32_t *nbr = d->mesh->nbr.as<int32_t>();
        DevBuf dist, flag, du, dkey, perm;
        JS_TRY(dist.alloc(N * 4, s));
        JS_TRY(flag.alloc(4, s));
        k_bdist_init<<<grid_for(N, 256, 152 * 32), 256, 0, s>>>(nbr, FS, N, nslab, dist.as<int32_t>());
        JS_LAUNCH_CHECK();
        for (int32_t r = 0; r < (int32_t)std::min<int64_t>(N, INT32_MAX - 1); ++r) {
            int changed = 0;
            JS_CUDA(cudaMemsetAsync(flag.p, 0, 4, s));
            k_bdist_step<<<grid_for(N, 256, 152 * 32), 256, 0, s>>>(nbr, FS, N, r, dist.as<int32_t>(), flag.as<int>());
            JS_LAUNCH_CHECK();
            JS_CUDA(cudaMemcpyAsync(&changed, flag.p, 4, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaStreamSynchronize(s));
            if (!changed) break;
        }
        int64_t n_dense = 0;
        {
            int64_t last_off = 0, last_cnt = 0;
            JS_CUDA(cudaMemcpyAsync(&last_off, uoff.as<int64_t>() + total - 1, 8, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaMemcpyAsync(&last_cnt, cnt.as<int64_t>() + total - 1, 8, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaStreamSynchronize(s));
            n_dense = last_off + last_cnt;
        }
        if (n_dense >= (1ll << 31)) {
            set_error("patch tasks: %lld units exceed the SLBD sort", (long long)n_dense);
            return JSWEEP_ERR_UNIMPLEMENTED;
        }
        JS_TRY(du.alloc((size_t)std::max<int64_t>(n_dense, 1) * 16, s));
        JS_TRY(dkey.alloc((size_t)std::max<int64_t>(n_dense, 1) * 4, s));
        JS_TRY(perm.alloc((size_t)std::max<int64_t>(n_dense, 1) * 4, s));
        k_patch_dense<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(
            d->s_order, d->s_lp, lpoff_d.as<int64_t>(), nlev_d.as<int32_t>(), tri_d.as<int64_t>(), M, N, nslab, U,
            total, uoff.as<int64_t>(), dist.as<int32_t>(), du.as<int4>(), dkey.as<uint32_t>());
        JS_LAUNCH_CHECK();
        if (n_dense > 0) {
            JS_TRY(radix_sort_segments(dkey.as<uint32_t>(), 1, n_dense, 32, nullptr, perm.as<int32_t>(), nullptr, s));
            k_patch_scatter<<<grid_for(n_dense, 256, 152 * 32), 256, 0, s>>>(
                du.as<int4>(), dkey.as<uint32_t>(), perm.as<int32_t>(), n_dense, uoff.as<int64_t>(),
                tri_d.as<int64_t>(), nlev_d.as<int32_t>(), M, nslab, W, ut.units.as<int4>());
            JS_LAUNCH_CHECK();
        }
        JS_CUDA(cudaStreamSynchronize(s));
    } else {
        k_patch_fill<<<grid_for(total, 256, 152 * 32), 256, 0, s>>>(d->s_order, d->s_lp, lpoff_d.as<int64_t>(),
                                                                    nlev_d.as<int32_t>(), tri_d.as<int64_t>(), M, N,
                                                                    nslab, U, total, uoff.as<int64_t>(), W,
                                                                    ut.units.as<int4>());
        JS_LAUNCH_CHECK();
        JS_CUDA(cudaStreamSynchronize(s));
    }
    ut.n_units = n_units;
    ut.warps = W;
    ut.slot_ptr.assign({0, n_units});
    ut.dirmajor = false;
    ut.mode = JSWEEP_MODE_PERSISTENT;
    ut.priority = prio;
    ut.cluster = U;
    ut.stagger = 0;
    ut.order = d->opt.unit_order;
    if (d->graph) {
        cudaGraphExecDestroy(d->graph);
        d->graph = nullptr;
        d->graph_key.clear();
    }
    return JSWEEP_OK;
}

// Direction-major table of the persistent schedule (see k_sweep_queue): every
// direction's units in layer order, with the direction boundaries.  Any
// priority other than patch tasks uses it (the order across directions is the
// warps' choice at run time; within a direction it is the depth order).
static int ensure_units_dir(Dags *d, int U, cudaStream_t s) {
    UnitTable &ut = d->ut;
    if (ut.dirmajor && ut.mode == JSWEEP_MODE_PERSISTENT && ut.cluster == U) return JSWEEP_OK;
    const int64_t M = d->M, Lmax = d->Smax;
    DevBuf ucnt, wscan, lpoff_d, nlev_d;
    JS_TRY(ucnt.alloc(M * Lmax * 8, s));
    JS_TRY(wscan.alloc(M * Lmax * 8, s));
    JS_TRY(lpoff_d.alloc((M + 1) * 8, s));
    JS_TRY(nlev_d.alloc(M * 4, s));
    std::vector<int32_t> nl32(M);
    for (int64_t m = 0; m < M; ++m) nl32[m] = (int32_t)d->slayers[m];
    JS_CUDA(cudaMemcpyAsync(lpoff_d.p, d->sp_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nlev_d.p, nl32.data(), M * 4, cudaMemcpyHostToDevice, s));
    k_unit_counts<<<grid_for(M * Lmax, 256, 4096), 256, 0, s>>>(d->s_lp, lpoff_d.as<int64_t>(),
                                                                nlev_d.as<int32_t>(), M, Lmax, U, ucnt.as<int64_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(scan_exclusive_i64(ucnt.as<int64_t>(), wscan.as<int64_t>(), M * Lmax, s));
    std::vector<int64_t> ws(M * Lmax), uc(1);
    JS_CUDA(cudaMemcpyAsync(ws.data(), wscan.p, M * Lmax * 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaMemcpyAsync(uc.data(), ucnt.as<int64_t>() + M * Lmax - 1, 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    const int64_t n_units = ws[M * Lmax - 1] + uc[0];
    std::vector<int64_t> dp(M + 1);
    for (int64_t m = 0; m < M; ++m) dp[m] = ws[m * Lmax];
    dp[M] = n_units;
    JS_TRY(ut.units.alloc(std::max<int64_t>(n_units, 1) * 16, s));
    JS_TRY(ut.dir_ptr.alloc((M + 1) * 8, s));
    JS_CUDA(cudaMemcpyAsync(ut.dir_ptr.p, dp.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    k_unit_fill_dir<<<grid_for(M * Lmax * 32, 256, 152 * 64), 256, 0, s>>>(d->s_lp, lpoff_d.as<int64_t>(),
                                                                  nlev_d.as<int32_t>(), ucnt.as<int64_t>(),
                                                                  wscan.as<int64_t>(), M, Lmax, U,
                                                                  ut.units.as<int4>());
    JS_LAUNCH_CHECK();
    JS_CUDA(cudaStreamSynchronize(s));
    ut.n_units = n_units;
    ut.warps = 0;
    ut.slot_ptr.assign({0, n_units});
    ut.dirmajor = true;
    ut.mode = JSWEEP_MODE_PERSISTENT;
    ut.priority = d->opt.priority;
    ut.cluster = U;
    ut.stagger = 0;
    ut.order = d->opt.unit_order;
    if (d->graph) {
        cudaGraphExecDestroy(d->graph);
        d->graph = nullptr;
        d->graph_key.clear();
    }
    return JSWEEP_OK;
}

int ensure_units(Dags *d, int mode, int max_cells, cudaStream_t s, int64_t resident_warps, bool dirmajor) {
    if (mode == JSWEEP_MODE_PATCH) return JSWEEP_OK;  // patch programs have their own schedule
    const int U = std::max(1, std::min(d->opt.cluster_cells, max_cells));
    int prio = d->opt.priority;
    if (patch_prio(prio) && mode != JSWEEP_MODE_PERSISTENT) prio = JSWEEP_PRIO_LEVEL;
    if (patch_prio(prio)) return ensure_units_patch(d, U, resident_warps, s, prio);
    if (dirmajor) return ensure_units_dir(d, U, s);
    int stagger = d->opt.octant_stagger > 0 ? d->opt.octant_stagger : (int)std::max<int64_t>(1, d->Smax / 4);
    if (prio != JSWEEP_PRIO_OCTANT) stagger = 0;
    const int order = d->opt.unit_order;
    UnitTable &ut = d->ut;
    if (!ut.dirmajor && ut.mode == mode && ut.priority == prio && ut.cluster == U && ut.stagger == stagger &&
        ut.order == order)
        return JSWEEP_OK;
    // schedule layers (levels or octant-aligned layers) play the part of levels here
    const int64_t M = d->M, Lmax = d->Smax;
    std::vector<int32_t> off(M, 0);
    for (int64_t m = 0; m < M; ++m) {
        if (prio == JSWEEP_PRIO_DEPTH) off[m] = (int32_t)(Lmax - d->slayers[m]);
        else if (prio == JSWEEP_PRIO_OCTANT) off[m] = (M % 8 == 0) ? (int32_t)((m / (M / 8)) * stagger) : 0;
    }
    int64_t Tmax = 0;
    for (int64_t m = 0; m < M; ++m) Tmax = std::max<int64_t>(Tmax, d->slayers[m] + off[m]);
    // directions grouped by octant (sign pattern), in increasing index inside a group
    std::vector<int32_t> oct(M), gmem, gstart(9, 0), gof(M), qpos(M);
    for (int64_t m = 0; m < M; ++m) {
        const double *o = d->quad->dirs.data() + 3 * m;
        oct[m] = (o[0] < 0 ? 1 : 0) | (o[1] < 0 ? 2 : 0) | (o[2] < 0 ? 4 : 0);
    }
    for (int g = 0; g < 8; ++g) {
        gstart[g] = (int32_t)gmem.size();
        for (int64_t m = 0; m < M; ++m)
            if (oct[m] == g) {
                qpos[m] = (int32_t)gmem.size();
                gof[m] = g;
                gmem.push_back((int32_t)m);
            }
    }
    gstart[8] = (int32_t)gmem.size();
    DevBuf ucnt, wscan, cnt2, base2, off_d, lpoff_d, nlev_d, gmem_d, gstart_d, gof_d, qpos_d;
    JS_TRY(gmem_d.alloc(M * 4, s));
    JS_TRY(gstart_d.alloc(9 * 4, s));
    JS_TRY(gof_d.alloc(M * 4, s));
    JS_TRY(qpos_d.alloc(M * 4, s));
    JS_CUDA(cudaMemcpyAsync(gmem_d.p, gmem.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(gstart_d.p, gstart.data(), 9 * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(gof_d.p, gof.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(qpos_d.p, qpos.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(ucnt.alloc(M * Lmax * 8, s));
    JS_TRY(wscan.alloc(M * Lmax * 8, s));
    JS_TRY(cnt2.alloc(Tmax * M * 8, s));
    JS_TRY(base2.alloc((Tmax * M + 1) * 8, s));
    JS_TRY(off_d.alloc(M * 4, s));
    JS_TRY(lpoff_d.alloc((M + 1) * 8, s));
    JS_TRY(nlev_d.alloc(M * 4, s));
    std::vector<int32_t> nl32(M);
    for (int64_t m = 0; m < M; ++m) nl32[m] = (int32_t)d->slayers[m];
    JS_CUDA(cudaMemcpyAsync(off_d.p, off.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(lpoff_d.p, d->sp_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nlev_d.p, nl32.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemsetAsync(cnt2.p, 0, Tmax * M * 8, s));
    k_unit_counts<<<grid_for(M * Lmax, 256, 4096), 256, 0, s>>>(d->s_lp, lpoff_d.as<int64_t>(),
                                                                nlev_d.as<int32_t>(), M, Lmax, U, ucnt.as<int64_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(scan_exclusive_i64(ucnt.as<int64_t>(), wscan.as<int64_t>(), M * Lmax, s));
    k_unit_slots<<<grid_for(M * Lmax, 256, 4096), 256, 0, s>>>(ucnt.as<int64_t>(), off_d.as<int32_t>(),
                                                               qpos_d.as<int32_t>(), M, Lmax, Tmax,
                                                               cnt2.as<int64_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(scan_exclusive_i64(cnt2.as<int64_t>(), base2.as<int64_t>(), Tmax * M, s));
    // total units = base2[last] + cnt2[last]
    int64_t last_base = 0, last_cnt = 0;
    JS_CUDA(cudaMemcpyAsync(&last_base, base2.as<int64_t>() + Tmax * M - 1, 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaMemcpyAsync(&last_cnt, cnt2.as<int64_t>() + Tmax * M - 1, 8, cudaMemcpyDeviceToHost, s));
    // slot boundaries (level-synchronous launches; merging of batched problems)
    std::vector<int64_t> b2h(Tmax * M);
    JS_CUDA(cudaMemcpyAsync(b2h.data(), base2.p, Tmax * M * 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    const int64_t n_units = last_base + last_cnt;
    JS_TRY(ut.units.alloc(std::max<int64_t>(n_units, 1) * 16, s));
    k_unit_fill<<<grid_for(M * Lmax * 32, 256, 152 * 64), 256, 0, s>>>(d->s_lp, lpoff_d.as<int64_t>(),
                                                              nlev_d.as<int32_t>(), ucnt.as<int64_t>(),
                                                              wscan.as<int64_t>(), base2.as<int64_t>(),
                                                              cnt2.as<int64_t>(), off_d.as<int32_t>(), M, Lmax, U,
                                                              gmem_d.as<int32_t>(), gstart_d.as<int32_t>(),
                                                              gof_d.as<int32_t>(), qpos_d.as<int32_t>(), order,
                                                              ut.units.as<int4>());
    JS_LAUNCH_CHECK();
    ut.slot_ptr.resize(Tmax + 1);
    for (int64_t t = 0; t < Tmax; ++t) ut.slot_ptr[t] = b2h[t * M];
    ut.slot_ptr[Tmax] = n_units;
    JS_CUDA(cudaStreamSynchronize(s));
    ut.n_units = n_units;
    ut.warps = 0;
    ut.dirmajor = false;
    ut.mode = mode;
    ut.priority = prio;
    ut.cluster = U;
    ut.stagger = stagger;
    ut.order = order;
    // the graph refers to the unit table
    if (d->graph) {
        cudaGraphExecDestroy(d->graph);
        d->graph = nullptr;
        d->graph_key.clear();
    }
    return JSWEEP_OK;
}

// dirs as [M][4] in the working precision
int ensure_dirs64x4(Dags *d, DevBuf &buf, cudaStream_t s) {
    if (buf.p) return JSWEEP_OK;
    std::vector<double> v(4 * d->M);
    for (int64_t m = 0; m < d->M; ++m) {
        for (int k = 0; k < 3; ++k) v[4 * m + k] = d->quad->dirs[3 * m + k];
        v[4 * m + 3] = 0.0;
    }
    JS_TRY(buf.alloc(v.size() * 8, s));
    JS_CUDA(cudaMemcpyAsync(buf.p, v.data(), v.size() * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaStreamSynchronize(s));
    return JSWEEP_OK;
}

namespace {

int resolve_mode(const Dags *d) {
    int mode = d->opt.sweep_mode;
    if (mode == JSWEEP_MODE_AUTO) mode = JSWEEP_MODE_LEVEL_SYNC;
    return mode;
}

// The persistent schedule of a single problem runs on the ready queues
// (k_sweep_queue) unless the face stream or the sweep-order psi is switched
// off or was refused, or the priority is patch tasks.
bool use_queues(const Dags *d, int mode) {
    return mode == JSWEEP_MODE_PERSISTENT && !patch_prio(d->opt.priority) && !d->opt.no_face_stream &&
           !d->opt.no_sweep_order_psi && !d->psi_seq_failed;
}

template <class T> SweepArgs<T> make_args(Dags *d, int Rp, bool has_inflow) {
    SweepArgs<T> a;
    a.N = d->N;
    a.M = (int)d->M;
    a.FS = d->mesh->FS;
    a.GS = d->mesh->GS;
    a.Fb = (int)d->mesh->Fb;
    a.order = d->s_order;
    a.mask = d->s_mask;
    if constexpr (sizeof(T) == 4) {
        a.geo = d->mesh->geo32.as<float4>();
        a.dirs = reinterpret_cast<const T *>(d->quad->dirs32.p);
    } else {
        a.geo = d->mesh->geo64.as<double4>();
        a.dirs = nullptr;  // set from the padded copy below
    }
    a.srcv = d->srcv.as<T>();
    a.inflow = has_inflow ? d->inflow.as<T>() : nullptr;
    a.psi = d->psi.as<T>();
    a.psi_seq = nullptr;  // set by the level-synchronous sweep when it uses the sweep-order copy
    a.psi_lag = d->psi_lag.as<T>();
    a.lag_ptr = d->lag_ptr.as<int32_t>();
    a.lag_face = d->lag_face.as<int32_t>();
    a.sface = d->mesh->sface.as<int32_t>();
    a.units = d->ut.units.as<int4>();
    a.bounds_err = bounds_word();
    (void)Rp;
    return a;
}

// Workspaces for (precision, padded rhs count).
int ensure_workspace(Dags *d, int prec, int Rp, int nrhs, cudaStream_t s) {
    const size_t es = prec == JSWEEP_F64 ? 8 : 4;
    const int64_t N = d->N, M = d->M;
    size_t before = (size_t)d->psi.p + (size_t)d->srcv.p + (size_t)d->inflow.p;
    JS_TRY(d->psi.ensure((size_t)M * N * Rp * es, s));
    const int RS = Rp >= 4 ? 2 * Rp : (Rp == 2 ? 4 : 2);  // src_stride
    JS_TRY(d->srcv.ensure((size_t)N * RS * es, s));
    JS_TRY(d->inflow.ensure((size_t)std::max<int64_t>(d->mesh->Fb, 1) * Rp * es, s));
    JS_TRY(d->phi_a.ensure((size_t)N * nrhs * es, s));
    JS_TRY(d->phi_b.ensure((size_t)N * nrhs * es, s));
    JS_TRY(d->red.ensure(64 * 8, s));
    JS_TRY(d->counters.ensure((size_t)(M + 8) * 8, s));
    if (d->lag_R != Rp || d->lag_prec != prec || !d->psi_lag.p) {
        JS_TRY(d->psi_lag.alloc((size_t)std::max<int64_t>(d->T, 1) * Rp * es, s));
        JS_CUDA(cudaMemsetAsync(d->psi_lag.p, 0, d->psi_lag.bytes, s));
        d->lag_R = Rp;
        d->lag_prec = prec;
    }
    size_t after = (size_t)d->psi.p + (size_t)d->srcv.p + (size_t)d->inflow.p;
    if (before != after && d->graph) {
        cudaGraphExecDestroy(d->graph);
        d->graph = nullptr;
        d->graph_key.clear();
    }
    return JSWEEP_OK;
}

template <class T, int R> constexpr int split_of() {
    return (int)(sizeof(T) * R / 16) > 1 ? (int)(sizeof(T) * R / 16) : 1;
}

template <class T, int R, int SPLIT, int MAXF, bool MG>
int launch_queue(Dags *d, const SweepArgs<T> &a, const unsigned char *coef, cudaStream_t s) {
    auto kern = k_sweep_queue<T, R, SPLIT, MAXF, MG>;
    int occ = 0;
    JS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarpsPerBlock * 32, 0));
    if (occ < 1) occ = 1;
    int bps = d->opt.blocks_per_sm;
    if (bps <= 0 || bps > occ) bps = occ;
    const int khz = device_clock_khz();
    const long long timeout = (long long)(d->opt.spin_timeout_s * (double)khz * 1000.0);
    int64_t grid = (int64_t)device_sm_count() * bps;
    const int64_t maxg = (d->ut.n_units + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > maxg) grid = std::max<int64_t>(1, maxg);
    // state: [0, 8) error word (read by check_sweep_error), then per direction a
    // cursor line and a counter line
    const size_t words = 8 + (size_t)2 * d->M * kQueueStride;
    JS_TRY(d->qstate.ensure(words * 4, s));
    int *st = d->qstate.as<int>();
    JS_CUDA(cudaMemsetAsync(st, 0, words * 4, s));
    JS_CUDA(cudaMemsetAsync(d->counters.p, 0, 8, s));
    unsigned *cursor = reinterpret_cast<unsigned *>(st + 8);
    int *done = st + 8 + (size_t)d->M * kQueueStride;
    int *err = reinterpret_cast<int *>(d->counters.p);
    kern<<<(unsigned)grid, kWarpsPerBlock * 32, 0, s>>>(a, d->ut.dir_ptr.as<int64_t>(), coef, cursor, done,
                                                         d->opt.debug_block_waits ? 1 : 0, err, timeout);
    JS_LAUNCH_CHECK();
    d->timing.sweep_launches = 1;
    return JSWEEP_OK;
}

template <class T, int R, int SPLIT, int MAXF>
int launch_dd(Dags *d, const SweepArgs<T> &a, cudaStream_t s) {
    auto kern = k_sweep_dd<T, R, SPLIT, MAXF>;
    int bps = d->opt.blocks_per_sm;
    int occ = 0;
    JS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarpsPerBlock * 32, 0));
    if (occ < 1) occ = 1;
    if (bps <= 0 || bps > occ) bps = occ;  // every warp must be resident
    const int khz = device_clock_khz();
    const long long timeout = (long long)(d->opt.spin_timeout_s * (double)khz * 1000.0);
    int64_t grid = (int64_t)device_sm_count() * bps;
    const int64_t maxg = (d->ut.n_units + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (grid > maxg) grid = std::max<int64_t>(1, maxg);
    if (patch_prio(d->ut.priority)) {
        // one warp per patch task: the table was laid out for exactly this many warps
        if (d->ut.warps > (int64_t)device_sm_count() * bps * kWarpsPerBlock) {
            set_error("patch tasks: %lld warps cannot all be resident", (long long)d->ut.warps);
            return JSWEEP_ERR_INVALID_ARG;
        }
        grid = d->ut.warps / kWarpsPerBlock;
    }
    // flags: one int per (direction, cell), stamped with the sweep epoch
    const size_t fbytes = (size_t)d->M * d->N * 4;
    if (!d->flags.p || d->flags.bytes < fbytes) {
        JS_TRY(d->flags.alloc(fbytes, s));
        JS_CUDA(cudaMemsetAsync(d->flags.p, 0, fbytes, s));
        d->epoch = 0;
    }
    if (d->epoch >= INT32_MAX - 2) {
        JS_CUDA(cudaMemsetAsync(d->flags.p, 0, fbytes, s));
        d->epoch = 0;
    }
    const int epoch = ++d->epoch;
    // debug_block_waits: wait for an epoch no sweep has written (test of the bounded-wait path)
    const int want = d->opt.debug_block_waits ? epoch + 1 : epoch;
    int *err = reinterpret_cast<int *>(d->counters.p);
    JS_CUDA(cudaMemsetAsync(err, 0, 8, s));
    kern<<<(unsigned)grid, kWarpsPerBlock * 32, 0, s>>>(a, d->ut.n_units, d->flags.as<int>(), epoch, want, err,
                                                         timeout);
    JS_LAUNCH_CHECK();
    d->timing.sweep_launches = 1;
    return JSWEEP_OK;
}

// Warps of the data-driven kernel that can be resident at once (patch tasks).
template <class T, int R> int64_t dd_resident_warps(const Dags *d) {
    constexpr int SPLIT = split_of<T, R>();
    const int FS = d->mesh->FS;
    const void *kern = FS <= 4 ? reinterpret_cast<const void *>(k_sweep_dd<T, R, SPLIT, 4>)
                     : FS <= 6 ? reinterpret_cast<const void *>(k_sweep_dd<T, R, SPLIT, 6>)
                               : reinterpret_cast<const void *>(k_sweep_dd<T, R, SPLIT, 7>);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarpsPerBlock * 32, 0) != cudaSuccess) occ = 1;
    int bps = d->opt.blocks_per_sm;
    if (occ < 1) occ = 1;
    if (bps <= 0 || bps > occ) bps = occ;
    return (int64_t)device_sm_count() * bps * kWarpsPerBlock;
}

template <class T, int R> int64_t patch_warps(const Dags *d, int mode) {
    return (mode == JSWEEP_MODE_PERSISTENT && patch_prio(d->opt.priority)) ? dd_resident_warps<T, R>(d) : 0;
}

// First slot of the tail: the slots from it to the end each hold fewer than
// tail_units units.  Returns the number of slots when there is no tail.  Only
// when slot t is layer t of every direction (JSWEEP_PRIO_LEVEL).
int64_t tail_slot(const Dags *d) {
    const auto &sp = d->ut.slot_ptr;
    const int64_t Tn = (int64_t)sp.size() - 1;
    if (d->opt.tail_units <= 0 || Tn <= 0 || d->ut.priority != JSWEEP_PRIO_LEVEL) return std::max<int64_t>(Tn, 0);
    const int64_t thr = d->opt.tail_units;
    int64_t S = Tn;
    while (S > 0 && sp[S] - sp[S - 1] < thr) --S;
    return S;
}

// Records the sweep's launches on the capture stream: one launch per slot
// before the tail slot S, then (S < number of slots) the tail, one block per
// direction.
template <class T, int R, int SPLIT, int MAXF, bool SEQ, bool MG>
void capture_levels(Dags *d, const SweepArgs<T> &a, cudaStream_t cs, const unsigned char *coef, int64_t S) {
    const auto &sp = d->ut.slot_ptr;
    const int64_t Tn = (int64_t)sp.size() - 1;
    bool first = true;
    for (int64_t l = 0; l < std::min(S, Tn); ++l) {
        const int64_t nu = sp[l + 1] - sp[l];
        if (nu <= 0) continue;
        const int64_t blocks = (nu + kLevelWarps - 1) / kLevelWarps;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)blocks);
        cfg.blockDim = dim3(kLevelWarps * 32);
        cfg.stream = cs;
        // slots after the first start early (programmatic dependent launch); the
        // first keeps a full dependency on whatever preceded the sweep
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = first ? 0 : 1;
        first = false;
        int64_t u0 = sp[l];
        if (coef) cudaLaunchKernelEx(&cfg, k_sweep_level_coef<T, R, SPLIT, MAXF, SEQ, MG>, a, u0, nu, coef);
        else cudaLaunchKernelEx(&cfg, k_sweep_level<T, R, SPLIT, MAXF>, a, u0, nu);
    }
    if (S < Tn) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)d->M);
        cfg.blockDim = dim3(kWarpsPerBlock * 32);
        cfg.stream = cs;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = first ? 0 : 1;
        cudaLaunchKernelEx(&cfg, k_sweep_tail<T, R, SPLIT, MAXF, SEQ, MG>, a, (const int32_t *)d->s_lp,
                           (const int64_t *)d->tail_lpoff.as<int64_t>(), (const int32_t *)d->tail_nlev.as<int32_t>(),
                           (int)S, coef);
    }
}

// The face-coefficient stream of the handle for precision T, built on first
// use (callers check the no_face_stream option), or nullptr when its
// allocation was refused (the sweep then reads the cell geometry).  It is
// built for the handle's sweep order and directions, which do not change
// after the build, so its address stays valid for the handle's life.
// positions: the variant whose interior neighbours are positions in the sweep
// order (read with the sweep-order copy of psi); it needs a temporary [M][N]
// int32 table of positions while it is filled.
template <class T>
const unsigned char *ensure_coef(Dags *d, const SweepArgs<T> &a, cudaStream_t s, bool positions = false) {
    Dags::FaceStream &fs = (positions ? d->pcoef : d->coef)[sizeof(T) == 8 ? 1 : 0];
    if (fs.failed) return nullptr;
    const int maxf = a.FS <= 4 ? 4 : a.FS <= 6 ? 6 : 7;
    if (fs.buf.p && fs.maxf == maxf && fs.order == d->s_order && fs.dirs == (const void *)a.dirs)
        return fs.buf.as<unsigned char>();
    const int rb = maxf == 4 ? coef_record_bytes<T, 4>() : maxf == 6 ? coef_record_bytes<T, 6>()
                                                                     : coef_record_bytes<T, 7>();
    if (fs.buf.alloc((size_t)d->N * d->M * rb, s) != JSWEEP_OK) {
        clear_error();
        fs.failed = true;
        return nullptr;
    }
    unsigned char *out = fs.buf.as<unsigned char>();
    const int grid = grid_for(d->N * d->M, 256, 152 * 64);
    DevBuf posbuf;
    const int32_t *pos = nullptr;
    if (positions) {
        if (posbuf.alloc((size_t)d->N * d->M * 4, s) != JSWEEP_OK) {
            clear_error();
            fs.buf.release();
            fs.failed = true;
            return nullptr;
        }
        k_sweep_positions<<<grid, 256, 0, s>>>(d->s_order, d->N, d->M, posbuf.as<int32_t>());
        note_launches(1);
        pos = posbuf.as<int32_t>();
    }
    if (maxf == 4) k_coef_fill<T, 4><<<grid, 256, 0, s>>>(d->s_order, a.geo, a.dirs, d->N, d->M, a.FS, a.GS, pos, out);
    else if (maxf == 6) k_coef_fill<T, 6><<<grid, 256, 0, s>>>(d->s_order, a.geo, a.dirs, d->N, d->M, a.FS, a.GS, pos, out);
    else k_coef_fill<T, 7><<<grid, 256, 0, s>>>(d->s_order, a.geo, a.dirs, d->N, d->M, a.FS, a.GS, pos, out);
    if (cudaGetLastError() != cudaSuccess) {
        fs.buf.release();
        fs.failed = true;
        return nullptr;
    }
    if (positions) cudaStreamSynchronize(s);  // the position table is released on return
    note_launches(1);
    fs.maxf = maxf;
    fs.order = d->s_order;
    fs.dirs = a.dirs;
    return out;
}

// MG: every right-hand side has its own sigma_t (see solve_cell_coef); only the
// face-stream schedules (level-synchronous, persistent queues) have it.
template <class T, int R, bool MG = false>
int sweep_core(Dags *d, SweepArgs<T> a, int mode, cudaStream_t s) {
    constexpr int SPLIT = split_of<T, R>();
    if (mode == JSWEEP_MODE_LEVEL_SYNC) {
        // default: the face stream with upwind positions and the sweep-order copy of
        // psi; else the face stream with upwind cell ids; else the cell geometry
        const unsigned char *coef = nullptr;
        if (!d->opt.no_face_stream && !d->opt.no_sweep_order_psi && !d->psi_seq_failed) {
            const size_t bytes = (size_t)d->M * d->N * R * sizeof(T);
            if (d->psi_seq.ensure(bytes, s) == JSWEEP_OK) {
                coef = ensure_coef<T>(d, a, s, true);
                if (coef) a.psi_seq = d->psi_seq.as<T>();
            } else {
                clear_error();
                d->psi_seq_failed = true;
            }
        }
        if (!coef && !d->opt.no_face_stream) coef = ensure_coef<T>(d, a, s);
        const bool seq = a.psi_seq != nullptr;
        if (MG && !coef) {
            set_error("per-group cross sections need the face stream");
            return JSWEEP_ERR_UNIMPLEMENTED;
        }
        const int64_t Tn = (int64_t)d->ut.slot_ptr.size() - 1;
        const int64_t S = coef ? tail_slot(d) : Tn;  // the tail runs on the face stream
        char key[512];
        snprintf(key, sizeof(key), "%d/%d/%d/%p/%p/%p/%p/%p/%p/%lld/%p/%lld/%p", (int)sizeof(T), R, (int)MG,
                 (const void *)a.srcv, (const void *)a.inflow, (const void *)a.psi, (const void *)a.psi_lag,
                 (const void *)a.units, (const void *)a.dirs, (long long)d->ut.n_units, (const void *)coef,
                 (long long)S, (const void *)a.psi_seq);
        if (!d->graph || d->graph_key != key) {
            if (d->graph) {
                cudaGraphExecDestroy(d->graph);
                d->graph = nullptr;
            }
            if (!d->capture_stream) JS_CUDA(cudaStreamCreateWithFlags(&d->capture_stream, cudaStreamNonBlocking));
            if (S < Tn) {
                // the tail kernel reads each direction's layer pointers and layer count
                const int64_t M = d->M;
                std::vector<int32_t> nl32(M);
                for (int64_t m = 0; m < M; ++m) nl32[m] = (int32_t)d->slayers[m];
                JS_TRY(d->tail_lpoff.ensure((size_t)(M + 1) * 8, s));
                JS_TRY(d->tail_nlev.ensure((size_t)M * 4, s));
                JS_CUDA(cudaMemcpyAsync(d->tail_lpoff.p, d->sp_off.data(), (size_t)(M + 1) * 8,
                                        cudaMemcpyHostToDevice, s));
                JS_CUDA(cudaMemcpyAsync(d->tail_nlev.p, nl32.data(), (size_t)M * 4, cudaMemcpyHostToDevice, s));
                JS_CUDA(cudaStreamSynchronize(s));
            }
            cudaStream_t cs = d->capture_stream;
            JS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            if (seq) {
                if (a.FS <= 4) capture_levels<T, R, SPLIT, 4, true, MG>(d, a, cs, coef, S);
                else if (a.FS <= 6) capture_levels<T, R, SPLIT, 6, true, MG>(d, a, cs, coef, S);
                else capture_levels<T, R, SPLIT, 7, true, MG>(d, a, cs, coef, S);
            } else {
                if (a.FS <= 4) capture_levels<T, R, SPLIT, 4, false, MG>(d, a, cs, coef, S);
                else if (a.FS <= 6) capture_levels<T, R, SPLIT, 6, false, MG>(d, a, cs, coef, S);
                else capture_levels<T, R, SPLIT, 7, false, MG>(d, a, cs, coef, S);
            }
            cudaGraph_t g;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (e != cudaSuccess) {
                set_error("graph capture failed: %s", cudaGetErrorString(e));
                return JSWEEP_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&d->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                set_error("graph instantiate failed: %s", cudaGetErrorString(e));
                d->graph = nullptr;
                return JSWEEP_ERR_CUDA;
            }
            d->graph_key = key;
        }
        JS_CUDA(cudaGraphLaunch(d->graph, s));
        int64_t nodes = S < Tn ? 1 : 0;
        for (int64_t l = 0; l < S; ++l) nodes += d->ut.slot_ptr[l + 1] > d->ut.slot_ptr[l];
        note_launches(nodes);
        d->timing.sweep_launches = nodes;
        return JSWEEP_OK;
    }
    if (mode == JSWEEP_MODE_PATCH && !MG) return launch_patch<T, R>(d, a, s);
    // persistent: the queue-driven kernel on the face stream with upwind positions
    // and the sweep-order copy of psi; per-cell epoch flags otherwise (and for
    // patch tasks, whose table is laid out for a fixed warp count)
    if (d->ut.dirmajor && use_queues(d, mode)) {
        const unsigned char *coef = nullptr;
        const size_t bytes = (size_t)d->M * d->N * R * sizeof(T);
        if (d->psi_seq.ensure(bytes, s) == JSWEEP_OK) {
            coef = ensure_coef<T>(d, a, s, true);
        } else {
            clear_error();
            d->psi_seq_failed = true;
        }
        if (coef) {
            a.psi_seq = d->psi_seq.as<T>();
            if (a.FS <= 4) return launch_queue<T, R, SPLIT, 4, MG>(d, a, coef, s);
            if (a.FS <= 6) return launch_queue<T, R, SPLIT, 6, MG>(d, a, coef, s);
            return launch_queue<T, R, SPLIT, 7, MG>(d, a, coef, s);
        }
    }
    if (MG) {
        set_error("per-group cross sections need the face stream");
        return JSWEEP_ERR_UNIMPLEMENTED;
    }
    if (a.FS <= 4) return launch_dd<T, R, SPLIT, 4>(d, a, s);
    if (a.FS <= 6) return launch_dd<T, R, SPLIT, 6>(d, a, s);
    return launch_dd<T, R, SPLIT, 7>(d, a, s);
}

int check_sweep_error(Dags *d, cudaStream_t s, int mode) {
    if (mode != JSWEEP_MODE_PERSISTENT && mode != JSWEEP_MODE_PATCH) return JSWEEP_OK;
    if (mode == JSWEEP_MODE_PATCH) JS_TRY(patch_counts(d, s));
    int err = 0;
    JS_CUDA(cudaMemcpyAsync(&err, d->counters.p, 4, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    if (err == 1) {
        set_error("persistent sweep: a dependency wait exceeded %.3g s", d->opt.spin_timeout_s);
        return JSWEEP_ERR_DEVICE_TIMEOUT;
    }
    if (err == 2) {
        set_error("patch programs: no progress for %.3g s", d->opt.spin_timeout_s);
        return JSWEEP_ERR_DEVICE_TIMEOUT;
    }
    if (err) {
        set_error("patch programs: the queue dispatched far more programs than the schedule needs");
        return JSWEEP_ERR_DEVICE_TIMEOUT;
    }
    return JSWEEP_OK;
}

template <class T, int R, bool MG = false>
int one_sweep(Dags *d, int mode, bool has_inflow, const T *wts, T *phi_dst, int nrhs, cudaStream_t s,
              const T *dirs_override) {
    SweepArgs<T> a = make_args<T>(d, R, has_inflow);
    if (dirs_override) a.dirs = dirs_override;
    JS_CUDA(cudaEventRecord(d->ev[0], s));
    JS_TRY((sweep_core<T, R, MG>(d, a, mode, s)));
    JS_CUDA(cudaEventRecord(d->ev[1], s));
    if (d->T > 0) {
        k_lag_update<T, R><<<grid_for(d->T, 256), 256, 0, s>>>(d->psi.as<T>(), d->lag_m.as<int32_t>(),
                                                              d->lag_up.as<int32_t>(), d->T, d->M, d->psi_lag.as<T>());
        JS_LAUNCH_CHECK();
    }
    JS_CUDA(cudaEventRecord(d->ev[2], s));
    k_phi<T, R><<<grid_for(d->N, 256, 152 * 16), 256, 0, s>>>(d->psi.as<T>(), wts, d->N, (int)d->M, nrhs, phi_dst);
    JS_LAUNCH_CHECK();
    JS_CUDA(cudaEventRecord(d->ev[3], s));
    return JSWEEP_OK;
}

}  // namespace

// The handle's face-coefficient stream for precision prec, built from the
// handle's own geometry and directions (the ones its sweeps and batches use),
// or nullptr when switched off or refused.  positions: the variant whose
// interior neighbours are positions in the handle's sweep order (read with a
// sweep-order copy of psi).
const unsigned char *ensure_face_stream(Dags *d, int prec, cudaStream_t s, bool positions) {
    if (prec == JSWEEP_F64) {
        if (ensure_dirs64x4(d, d->dirs4_64, s) != JSWEEP_OK) {
            clear_error();
            return nullptr;
        }
        SweepArgs<double> a{};
        a.FS = d->mesh->FS;
        a.GS = d->mesh->GS;
        a.geo = d->mesh->geo64.as<double4>();
        a.dirs = d->dirs4_64.as<double>();
        return ensure_coef<double>(d, a, s, positions);
    }
    SweepArgs<float> a{};
    a.FS = d->mesh->FS;
    a.GS = d->mesh->GS;
    a.geo = d->mesh->geo32.as<float4>();
    a.dirs = reinterpret_cast<const float *>(d->quad->dirs32.p);
    return ensure_coef<float>(d, a, s, positions);
}

// FP64 directions in [M][4] layout (the FP32 copy lives in the quadrature).
static int dirs64x4(Dags *d, cudaStream_t s, const double **out) {
    JS_TRY(ensure_dirs64x4(d, d->dirs4_64, s));
    *out = d->dirs4_64.as<double>();
    return JSWEEP_OK;
}

template <class T, int R>
static int run_sweep_t(Dags *d, int nrhs, const void *sigma_t, const void *ang_source, const void *inflow,
                       void *phi_out, void *psi_out, cudaStream_t s) {
    const int mode = resolve_mode(d);
    JS_TRY(ensure_units(d, mode, 32 / split_of<T, R>(), s, patch_warps<T, R>(d, mode), use_queues(d, mode)));
    JS_TRY(ensure_workspace(d, sizeof(T) == 8 ? JSWEEP_F64 : JSWEEP_F32, R, nrhs, s));
    const T *vol = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->mesh->vol64.p)
                                  : reinterpret_cast<const T *>(d->mesh->vol32.p);
    const T *w = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->quad->w64.p)
                                : reinterpret_cast<const T *>(d->quad->w32.p);
    const double *d64 = nullptr;
    if (sizeof(T) == 8) JS_TRY(dirs64x4(d, s, &d64));
    k_source_prep<T, R><<<grid_for(d->N, 256, 152 * 16), 256, 0, s>>>(
        (const T *)sigma_t, (const T *)ang_source, vol, d->N, nrhs, d->srcv.as<T>());
    JS_LAUNCH_CHECK();
    const bool has_inflow = inflow != nullptr;
    if (has_inflow) {
        const size_t es = sizeof(T);
        JS_CUDA(cudaMemsetAsync(d->inflow.p, 0, d->inflow.bytes, s));
        JS_CUDA(cudaMemcpyAsync(d->inflow.p, inflow, (size_t)nrhs * d->mesh->Fb * es, cudaMemcpyDeviceToDevice, s));
    }
    JS_TRY((one_sweep<T, R>(d, mode, has_inflow, w, (T *)phi_out, nrhs, s, (const T *)d64)));
    if (psi_out) {
        k_psi_out<T, R><<<grid_for(d->N * d->M, 256, 152 * 32), 256, 0, s>>>(d->psi.as<T>(), d->N, (int)d->M, nrhs,
                                                                            (T *)psi_out);
        JS_LAUNCH_CHECK();
    }
    JS_TRY(check_sweep_error(d, s, mode));
    JS_CUDA(cudaStreamSynchronize(s));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, d->ev[0], d->ev[1]);
    cudaEventElapsedTime(&b, d->ev[2], d->ev[3]);
    d->timing.sweep_ms = a;
    d->timing.phi_ms = b;
    return JSWEEP_OK;
}

template <class T, int R>
static int run_si_t(Dags *d, int nrhs, const void *sigma_t, const void *c_ratio, const void *q, const void *inflow,
                    double tol, int max_iters, void *phi_out, int *iters_out, double *resid_out, cudaStream_t s) {
    const int mode = resolve_mode(d);
    JS_TRY(ensure_units(d, mode, 32 / split_of<T, R>(), s, patch_warps<T, R>(d, mode), use_queues(d, mode)));
    JS_TRY(ensure_workspace(d, sizeof(T) == 8 ? JSWEEP_F64 : JSWEEP_F32, R, nrhs, s));
    JS_CUDA(cudaMemsetAsync(d->psi_lag.p, 0, d->psi_lag.bytes, s));
    const T *vol = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->mesh->vol64.p)
                                  : reinterpret_cast<const T *>(d->mesh->vol32.p);
    const T *w = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->quad->w64.p)
                                : reinterpret_cast<const T *>(d->quad->w32.p);
    const double *d64 = nullptr;
    if (sizeof(T) == 8) JS_TRY(dirs64x4(d, s, &d64));
    const bool has_inflow = inflow != nullptr;
    if (has_inflow) {
        JS_CUDA(cudaMemsetAsync(d->inflow.p, 0, d->inflow.bytes, s));
        JS_CUDA(cudaMemcpyAsync(d->inflow.p, inflow, (size_t)nrhs * d->mesh->Fb * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    T *phi_old = nullptr;  // phi^0 = 0
    T *bufs[2] = {d->phi_a.as<T>(), d->phi_b.as<T>()};
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(d->red.p);
    double *resid_d = reinterpret_cast<double *>(acc + 32);
    double resid_h[9] = {0};
    int it = 0;
    bool conv = false;
    T *phi_new = bufs[0];
    for (it = 1; it <= max_iters; ++it) {
        phi_new = bufs[(it - 1) & 1];
        k_emission<T, R><<<grid_for(d->N, 256, 152 * 16), 256, 0, s>>>(
            (const T *)sigma_t, (const T *)c_ratio, (const T *)q, phi_old, vol, d->N, nrhs, d->srcv.as<T>());
        JS_LAUNCH_CHECK();
        JS_TRY((one_sweep<T, R>(d, mode, has_inflow, w, phi_new, nrhs, s, (const T *)d64)));
        JS_CUDA(cudaMemsetAsync(acc, 0, 2 * 8 * 8, s));
        k_resid<T><<<dim3(grid_for(d->N, 256, 152 * 4), nrhs), 256, 0, s>>>(phi_new, phi_old, d->N, acc);
        JS_LAUNCH_CHECK();
        k_resid_final<<<1, 32, 0, s>>>(acc, nrhs, resid_d);
        JS_LAUNCH_CHECK();
        JS_CUDA(cudaMemcpyAsync(resid_h, resid_d, (nrhs + 1) * 8, cudaMemcpyDeviceToHost, s));
        JS_CUDA(cudaStreamSynchronize(s));
        JS_TRY(check_sweep_error(d, s, mode));
        phi_old = phi_new;
        if (resid_h[nrhs] < tol) {
            conv = true;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    JS_CUDA(cudaMemcpyAsync(phi_out, phi_new, (size_t)nrhs * d->N * sizeof(T), cudaMemcpyDeviceToDevice, s));
    JS_CUDA(cudaStreamSynchronize(s));
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, d->ev[0], d->ev[1]);
    cudaEventElapsedTime(&b, d->ev[2], d->ev[3]);
    d->timing.sweep_ms = a;
    d->timing.phi_ms = b;
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = resid_h[nrhs];
    if (!conv) {
        set_error("source iteration did not reach tol %g in %d iterations (residual %g)", tol, max_iters,
                  resid_h[nrhs]);
        return JSWEEP_ERR_NOT_CONVERGED;
    }
    return JSWEEP_OK;
}

// Multigroup source iteration (the appendix's transport equation over energy
// groups, Alg. 1): phi^0 = 0; each iteration forms every group's source from
// the previous iterate of all groups (k_emission_mg), then sweeps the groups
// one after the other as single-rhs sweeps with their own sigma_t, and stops
// when every group's relative max-norm change is below tol.  The groups share
// the handle's psi, source-record, inflow and lagged-value buffers (so the
// captured level-synchronous graph serves all of them): a group's inflow and
// lagged values are copied in before its sweep and its lagged values copied
// out after it.
// The same iteration with the G <= 8 groups riding the right-hand-side
// dimension: one sweep per iteration carries every group (per-group sigma_t in
// the source records, per-group lagged values and inflow rows), on the
// schedules that read the face stream.  Each group is solved by the same
// operations as in a one-rhs sweep, so the results are those of the
// group-by-group iteration, bit for bit.
template <class T, int R>
static int run_si_mg_groups_t(Dags *d, int G, const void *sigma_t, const void *sigma_s, const void *q,
                              const void *inflow, double tol, int max_iters, void *phi_out, int *iters_out,
                              double *resid_out, cudaStream_t s) {
    const int mode = resolve_mode(d);
    JS_TRY(ensure_units(d, mode, 32 / split_of<T, R>(), s, 0, use_queues(d, mode)));
    JS_TRY(ensure_workspace(d, sizeof(T) == 8 ? JSWEEP_F64 : JSWEEP_F32, R, G, s));
    JS_CUDA(cudaMemsetAsync(d->psi_lag.p, 0, d->psi_lag.bytes, s));
    const int64_t N = d->N, Fb = d->mesh->Fb;
    const size_t es = sizeof(T);
    const T *vol = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->mesh->vol64.p)
                                  : reinterpret_cast<const T *>(d->mesh->vol32.p);
    const T *w = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->quad->w64.p)
                                : reinterpret_cast<const T *>(d->quad->w32.p);
    const double *d64 = nullptr;
    if (sizeof(T) == 8) JS_TRY(dirs64x4(d, s, &d64));
    const bool has_inflow = inflow != nullptr;
    if (has_inflow) {
        JS_CUDA(cudaMemsetAsync(d->inflow.p, 0, d->inflow.bytes, s));
        JS_CUDA(cudaMemcpyAsync(d->inflow.p, inflow, (size_t)G * Fb * es, cudaMemcpyDeviceToDevice, s));
    }
    DevBuf src_d;
    const int rc = [&]() -> int {
        JS_TRY(src_d.alloc((size_t)G * N * es, s));
        T *bufs[2] = {d->phi_a.as<T>(), d->phi_b.as<T>()};
        T *phi_old = nullptr;  // phi^0 = 0
        T *phi_new = bufs[0];
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(d->red.p);
        double *resid_d = reinterpret_cast<double *>(acc + 32);
        double resid_h[9] = {0};
        int it = 0;
        bool conv = false;
        for (it = 1; it <= max_iters; ++it) {
            phi_new = bufs[(it - 1) & 1];
            k_emission_mg<T><<<grid_for((int64_t)G * N, 256, 152 * 16), 256, 0, s>>>(
                (const T *)sigma_s, (const T *)q, phi_old, N, G, src_d.as<T>());
            JS_LAUNCH_CHECK();
            k_source_prep_mg<T, R><<<grid_for(N, 256, 152 * 16), 256, 0, s>>>((const T *)sigma_t, src_d.as<T>(), vol,
                                                                             N, G, d->srcv.as<T>());
            JS_LAUNCH_CHECK();
            JS_TRY((one_sweep<T, R, true>(d, mode, has_inflow, w, phi_new, G, s, (const T *)d64)));
            JS_CUDA(cudaMemsetAsync(acc, 0, 2 * 8 * 8, s));
            k_resid<T><<<dim3(grid_for(N, 256, 152 * 4), G), 256, 0, s>>>(phi_new, phi_old, N, acc);
            JS_LAUNCH_CHECK();
            k_resid_final<<<1, 32, 0, s>>>(acc, G, resid_d);
            JS_LAUNCH_CHECK();
            JS_CUDA(cudaMemcpyAsync(resid_h, resid_d, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaStreamSynchronize(s));
            JS_TRY(check_sweep_error(d, s, mode));
            phi_old = phi_new;
            if (resid_h[G] < tol) {
                conv = true;
                break;
            }
        }
        if (it > max_iters) it = max_iters;
        JS_CUDA(cudaMemcpyAsync(phi_out, phi_new, (size_t)G * N * es, cudaMemcpyDeviceToDevice, s));
        // the handle's lagged values belong to the groups: start later sweeps from 0
        JS_CUDA(cudaMemsetAsync(d->psi_lag.p, 0, d->psi_lag.bytes, s));
        JS_CUDA(cudaStreamSynchronize(s));
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, d->ev[0], d->ev[1]);
        cudaEventElapsedTime(&b, d->ev[2], d->ev[3]);
        d->timing.sweep_ms = a;
        d->timing.phi_ms = b;
        if (iters_out) *iters_out = it;
        if (resid_out) *resid_out = resid_h[G];
        if (!conv) {
            set_error("multigroup source iteration did not reach tol %g in %d iterations (residual %g)", tol,
                      max_iters, resid_h[G]);
            return JSWEEP_ERR_NOT_CONVERGED;
        }
        return JSWEEP_OK;
    }();
    cudaStreamSynchronize(s);
    return rc;
}

template <class T>
static int run_si_mg_t(Dags *d, int G, const void *sigma_t, const void *sigma_s, const void *q, const void *inflow,
                       double tol, int max_iters, void *phi_out, int *iters_out, double *resid_out, cudaStream_t s) {
    const int mode = resolve_mode(d);
    // groups ride the right-hand sides where the schedule reads the face stream
    const bool fast = G <= 8 && !d->opt.no_face_stream &&
                      (mode == JSWEEP_MODE_LEVEL_SYNC || use_queues(d, mode));
    if (fast) {
        switch (pad_rhs(G)) {
            case 1: return run_si_mg_groups_t<T, 1>(d, G, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out,
                                                     iters_out, resid_out, s);
            case 2: return run_si_mg_groups_t<T, 2>(d, G, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out,
                                                     iters_out, resid_out, s);
            case 4: return run_si_mg_groups_t<T, 4>(d, G, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out,
                                                     iters_out, resid_out, s);
            default: return run_si_mg_groups_t<T, 8>(d, G, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out,
                                                      iters_out, resid_out, s);
        }
    }
    JS_TRY(ensure_units(d, mode, 32 / split_of<T, 1>(), s, patch_warps<T, 1>(d, mode), use_queues(d, mode)));
    JS_TRY(ensure_workspace(d, sizeof(T) == 8 ? JSWEEP_F64 : JSWEEP_F32, 1, 1, s));
    const int64_t N = d->N, Fb = d->mesh->Fb, Tl = d->T;
    const size_t es = sizeof(T);
    const T *vol = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->mesh->vol64.p)
                                  : reinterpret_cast<const T *>(d->mesh->vol32.p);
    const T *w = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->quad->w64.p)
                                : reinterpret_cast<const T *>(d->quad->w32.p);
    const double *d64 = nullptr;
    if (sizeof(T) == 8) JS_TRY(dirs64x4(d, s, &d64));
    DevBuf src_d, phi_d0, phi_d1, lag_d;
    // the loop runs in a lambda so that every exit, error or not, waits for the
    // stream before the local buffers above are released
    const int rc = [&]() -> int {
        JS_TRY(src_d.alloc((size_t)G * N * es, s));
        JS_TRY(phi_d0.alloc((size_t)G * N * es, s));
        JS_TRY(phi_d1.alloc((size_t)G * N * es, s));
        JS_TRY(lag_d.alloc((size_t)G * std::max<int64_t>(Tl, 1) * es, s));
        JS_CUDA(cudaMemsetAsync(lag_d.p, 0, lag_d.bytes, s));
        const bool has_inflow = inflow != nullptr;
        T *bufs[2] = {phi_d0.as<T>(), phi_d1.as<T>()};
        T *phi_old = nullptr;  // phi^0 = 0
        T *phi_new = bufs[0];
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(d->red.p);
        double *resid_d = reinterpret_cast<double *>(acc + 32);
        double resid_h[9] = {0};
        int it = 0;
        bool conv = false;
        for (it = 1; it <= max_iters; ++it) {
            phi_new = bufs[(it - 1) & 1];
            k_emission_mg<T><<<grid_for((int64_t)G * N, 256, 152 * 16), 256, 0, s>>>(
                (const T *)sigma_s, (const T *)q, phi_old, N, G, src_d.as<T>());
            JS_LAUNCH_CHECK();
            for (int g = 0; g < G; ++g) {
                k_source_prep<T, 1><<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(
                    (const T *)sigma_t + (int64_t)g * N, src_d.as<T>() + (int64_t)g * N, vol, N, 1, d->srcv.as<T>());
                JS_LAUNCH_CHECK();
                if (has_inflow && Fb > 0)
                    JS_CUDA(cudaMemcpyAsync(d->inflow.p, (const T *)inflow + (int64_t)g * Fb, (size_t)Fb * es,
                                            cudaMemcpyDeviceToDevice, s));
                if (Tl > 0)
                    JS_CUDA(cudaMemcpyAsync(d->psi_lag.p, lag_d.as<T>() + (int64_t)g * Tl, (size_t)Tl * es,
                                            cudaMemcpyDeviceToDevice, s));
                JS_TRY((one_sweep<T, 1>(d, mode, has_inflow, w, phi_new + (int64_t)g * N, 1, s, (const T *)d64)));
                JS_TRY(check_sweep_error(d, s, mode));  // the next group's launch clears the error flag
                if (Tl > 0)
                    JS_CUDA(cudaMemcpyAsync(lag_d.as<T>() + (int64_t)g * Tl, d->psi_lag.p, (size_t)Tl * es,
                                            cudaMemcpyDeviceToDevice, s));
            }
            JS_CUDA(cudaMemsetAsync(acc, 0, 2 * 8 * 8, s));
            k_resid<T><<<dim3(grid_for(N, 256, 152 * 4), G), 256, 0, s>>>(phi_new, phi_old, N, acc);
            JS_LAUNCH_CHECK();
            k_resid_final<<<1, 32, 0, s>>>(acc, G, resid_d);
            JS_LAUNCH_CHECK();
            JS_CUDA(cudaMemcpyAsync(resid_h, resid_d, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost, s));
            JS_CUDA(cudaStreamSynchronize(s));
            phi_old = phi_new;
            if (resid_h[G] < tol) {
                conv = true;
                break;
            }
        }
        if (it > max_iters) it = max_iters;
        JS_CUDA(cudaMemcpyAsync(phi_out, phi_new, (size_t)G * N * es, cudaMemcpyDeviceToDevice, s));
        // the handle's lagged values belonged to the last group: start later sweeps from 0
        JS_CUDA(cudaMemsetAsync(d->psi_lag.p, 0, d->psi_lag.bytes, s));
        JS_CUDA(cudaStreamSynchronize(s));
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, d->ev[0], d->ev[1]);
        cudaEventElapsedTime(&b, d->ev[2], d->ev[3]);
        d->timing.sweep_ms = a;
        d->timing.phi_ms = b;
        if (iters_out) *iters_out = it;
        if (resid_out) *resid_out = resid_h[G];
        if (!conv) {
            set_error("multigroup source iteration did not reach tol %g in %d iterations (residual %g)", tol,
                      max_iters, resid_h[G]);
            return JSWEEP_ERR_NOT_CONVERGED;
        }
        return JSWEEP_OK;
    }();
    cudaStreamSynchronize(s);
    return rc;
}

int run_source_iteration_mg(Dags *d, int n_groups, int prec, const void *sigma_t, const void *sigma_s,
                            const void *q, const void *inflow, double tol, int max_iters, void *phi_out,
                            int *iters_out, double *resid_out, cudaStream_t s) {
    if (prec == JSWEEP_F64)
        return run_si_mg_t<double>(d, n_groups, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out, iters_out,
                                   resid_out, s);
    return run_si_mg_t<float>(d, n_groups, sigma_t, sigma_s, q, inflow, tol, max_iters, phi_out, iters_out,
                              resid_out, s);
}

int run_sweep(Dags *d, int nrhs, int prec, const void *sigma_t, const void *ang_source, const void *inflow,
              void *phi_out, void *psi_out, cudaStream_t s) {
    const int Rp = pad_rhs(nrhs);
    if (prec == JSWEEP_F64) {
        switch (Rp) {
            case 1: return run_sweep_t<double, 1>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
            case 2: return run_sweep_t<double, 2>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
            case 4: return run_sweep_t<double, 4>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
            default: return run_sweep_t<double, 8>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
        }
    }
    switch (Rp) {
        case 1: return run_sweep_t<float, 1>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
        case 2: return run_sweep_t<float, 2>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
        case 4: return run_sweep_t<float, 4>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
        default: return run_sweep_t<float, 8>(d, nrhs, sigma_t, ang_source, inflow, phi_out, psi_out, s);
    }
}

int run_source_iteration(Dags *d, int nrhs, int prec, const void *sigma_t, const void *c_ratio, const void *q,
                         const void *inflow, double tol, int max_iters, void *phi_out, int *iters_out,
                         double *resid_out, cudaStream_t s) {
    const int Rp = pad_rhs(nrhs);
#define JS_SI(T, R) run_si_t<T, R>(d, nrhs, sigma_t, c_ratio, q, inflow, tol, max_iters, phi_out, iters_out, resid_out, s)
    if (prec == JSWEEP_F64) {
        switch (Rp) {
            case 1: return JS_SI(double, 1);
            case 2: return JS_SI(double, 2);
            case 4: return JS_SI(double, 4);
            default: return JS_SI(double, 8);
        }
    }
    switch (Rp) {
        case 1: return JS_SI(float, 1);
        case 2: return JS_SI(float, 2);
        case 4: return JS_SI(float, 4);
        default: return JS_SI(float, 8);
    }
#undef JS_SI
}

// ---- source iteration without device allocations ----------------------------------
// Some callers cannot allocate device memory once they are running: for example
// a host application that hands this library a device whose memory is entirely
// owned and budgeted by its own runtime, or a latency-critical solve loop in
// which the device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable.  jsweep_source_iterate_noalloc serves them: every temporary it
// needs lives in one fixed, file-scope device array (kNoallocScratchBytes),
// which every GPU that loads this library holds until the process exits.
constexpr size_t kNoallocScratchBytes = JSWEEP_NOALLOC_SCRATCH_BYTES;

namespace {

// Sweep of one level for every direction, reading the level pointers directly
// (no work-unit table, which would have to be allocated).
template <class T, int R, int SPLIT, int MAXF>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_sweep_level_na(SweepArgs<T> a, const int32_t *lp, const int64_t *lp_off, const int64_t *nlev, int32_t l) {
    const int64_t m = blockIdx.y;
    if (l >= nlev[m]) return;
    const int32_t p0 = lp[lp_off[m] + l], p1 = lp[lp_off[m] + l + 1];
    constexpr int CPW = 32 / SPLIT;
    const int lane = threadIdx.x & 31, cell = lane / SPLIT, sub = lane % SPLIT;
    const int32_t wid = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int32_t stride = gridDim.x * kWarpsPerBlock * CPW;
    for (int32_t pos = p0 + wid * CPW + cell; pos < p1; pos += stride) {
        if (!JS_IN_RANGE(a, pos, a.N, 4)) continue;
        const int64_t idx = m * a.N + pos;
        solve_cell<T, R, SPLIT, MAXF, false>(a, (int)m, __ldg(a.order + idx), __ldg(a.mask + idx), sub, nullptr, 0,
                                             nullptr, 0);
    }
}

__global__ void k_pad_dirs(const double *d3, int64_t M, double *d4) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        d4[4 * m] = d3[3 * m];
        d4[4 * m + 1] = d3[3 * m + 1];
        d4[4 * m + 2] = d3[3 * m + 2];
        d4[4 * m + 3] = 0.0;
    }
}

}  // namespace

}  // namespace js

// The scratch array (file scope, internal linkage).
static __device__ __align__(256) unsigned char g_noalloc_scratch[js::kNoallocScratchBytes];

namespace js {
namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device: looked up once
// per device, with that device current.
int noalloc_scratch(void **out) {
    int dev = 0;
    JS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal %d not supported", dev);
        return JSWEEP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
            return JSWEEP_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return JSWEEP_OK;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T, int R>
int si_noalloc_t(Dags *d, int nrhs, const void *sigma_t, const void *c_ratio, const void *q, const void *inflow,
                 double tol, int max_iters, void *phi_out, int *iters_out, double *resid_out, cudaStream_t s) {
    constexpr int SPLIT = split_of<T, R>();
    const int64_t N = d->N, M = d->M;
    const int64_t Tl = std::max<int64_t>(d->T, 1);
    // scratch layout
    size_t off = 0;
    const size_t o_psi = off;   off = align256(off + (size_t)M * N * R * sizeof(T));
    const size_t o_src = off;   off = align256(off + (size_t)N * src_stride<R>() * sizeof(T));
    const size_t o_lag = off;   off = align256(off + (size_t)Tl * R * sizeof(T));
    const size_t o_phi0 = off;  off = align256(off + (size_t)nrhs * N * sizeof(T));
    const size_t o_phi1 = off;  off = align256(off + (size_t)nrhs * N * sizeof(T));
    const size_t o_inf = off;   off = align256(off + (size_t)std::max<int64_t>(d->mesh->Fb, 1) * R * sizeof(T));
    const size_t o_dirs = off;  off = align256(off + (size_t)M * 4 * sizeof(double));
    const size_t o_lpoff = off; off = align256(off + (size_t)(M + 1) * 8);
    const size_t o_nlev = off;  off = align256(off + (size_t)M * 8);
    const size_t o_acc = off;   off = align256(off + 32 * 8 + 16 * 8);
    if (off > kNoallocScratchBytes) {
        set_error("jsweep_source_iterate_noalloc: this problem needs %zu bytes of scratch, more than the %zu-byte "
                  "fixed array (directions x cells x right-hand sides is too large)",
                  off, kNoallocScratchBytes);
        return JSWEEP_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    JS_TRY(noalloc_scratch(&base));
    char *b = static_cast<char *>(base);
    T *psi = reinterpret_cast<T *>(b + o_psi);
    T *srcv = reinterpret_cast<T *>(b + o_src);
    T *lag = reinterpret_cast<T *>(b + o_lag);
    T *phis[2] = {reinterpret_cast<T *>(b + o_phi0), reinterpret_cast<T *>(b + o_phi1)};
    T *infl = reinterpret_cast<T *>(b + o_inf);
    double *d4 = reinterpret_cast<double *>(b + o_dirs);
    int64_t *lpoff = reinterpret_cast<int64_t *>(b + o_lpoff);
    int64_t *nlev = reinterpret_cast<int64_t *>(b + o_nlev);
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(b + o_acc);
    double *resid_d = reinterpret_cast<double *>(acc + 32);

    // what must start at zero: the lagged values (and the padded inflow rows)
    JS_CUDA(cudaMemsetAsync(lag, 0, (size_t)Tl * R * sizeof(T), s));
    if (inflow) {
        JS_CUDA(cudaMemsetAsync(infl, 0, (size_t)std::max<int64_t>(d->mesh->Fb, 1) * R * sizeof(T), s));
        JS_CUDA(cudaMemcpyAsync(infl, inflow, (size_t)nrhs * d->mesh->Fb * sizeof(T), cudaMemcpyDeviceToDevice, s));
    }
    JS_CUDA(cudaMemcpyAsync(lpoff, d->lp_off.data(), (M + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nlev, d->nlevels.data(), M * 8, cudaMemcpyHostToDevice, s));
    SweepArgs<T> a;
    a.N = N;
    a.M = (int)M;
    a.FS = d->mesh->FS;
    a.GS = d->mesh->GS;
    a.Fb = (int)d->mesh->Fb;
    a.order = d->order.as<int32_t>();
    a.mask = d->mask.as<uint8_t>();
    if constexpr (sizeof(T) == 4) {
        a.geo = d->mesh->geo32.as<float4>();
        a.dirs = reinterpret_cast<const T *>(d->quad->dirs32.p);
    } else {
        a.geo = d->mesh->geo64.as<double4>();
        k_pad_dirs<<<grid_for(M, 256), 256, 0, s>>>(d->quad->dirs64.as<double>(), M, d4);
        JS_LAUNCH_CHECK();
        a.dirs = reinterpret_cast<const T *>(d4);
    }
    a.srcv = srcv;
    a.inflow = inflow ? infl : nullptr;
    a.psi = psi;
    a.psi_seq = nullptr;
    a.psi_lag = lag;
    a.lag_ptr = d->lag_ptr.as<int32_t>();
    a.lag_face = d->lag_face.as<int32_t>();
    a.sface = d->mesh->sface.as<int32_t>();
    a.units = nullptr;
    a.bounds_err = bounds_word();
    const T *vol = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->mesh->vol64.p)
                                  : reinterpret_cast<const T *>(d->mesh->vol32.p);
    const T *w = sizeof(T) == 8 ? reinterpret_cast<const T *>(d->quad->w64.p)
                                : reinterpret_cast<const T *>(d->quad->w32.p);
    const int gx = (int)std::min<int64_t>(std::max<int64_t>(1, N / (kWarpsPerBlock * (32 / SPLIT) * 16)), 32);
    T *phi_old = nullptr, *phi_new = phis[0];
    double resid_h[9] = {0};
    bool conv = false;
    int it = 0;
    for (it = 1; it <= max_iters; ++it) {
        phi_new = phis[(it - 1) & 1];
        k_emission<T, R><<<grid_for(N, 256, 152 * 16), 256, 0, s>>>((const T *)sigma_t, (const T *)c_ratio,
                                                                    (const T *)q, phi_old, vol, N, nrhs, srcv);
        JS_LAUNCH_CHECK();
        for (int64_t l = 0; l < d->Lmax; ++l) {
            if (a.FS <= 4)
                k_sweep_level_na<T, R, SPLIT, 4><<<dim3(gx, (unsigned)M), kWarpsPerBlock * 32, 0, s>>>(
                    a, d->lp.as<int32_t>(), lpoff, nlev, (int32_t)l);
            else if (a.FS <= 6)
                k_sweep_level_na<T, R, SPLIT, 6><<<dim3(gx, (unsigned)M), kWarpsPerBlock * 32, 0, s>>>(
                    a, d->lp.as<int32_t>(), lpoff, nlev, (int32_t)l);
            else
                k_sweep_level_na<T, R, SPLIT, 7><<<dim3(gx, (unsigned)M), kWarpsPerBlock * 32, 0, s>>>(
                    a, d->lp.as<int32_t>(), lpoff, nlev, (int32_t)l);
            JS_LAUNCH_CHECK();
        }
        if (d->T > 0) {
            k_lag_update<T, R><<<grid_for(d->T, 256), 256, 0, s>>>(psi, d->lag_m.as<int32_t>(), d->lag_up.as<int32_t>(),
                                                                  d->T, M, lag);
            JS_LAUNCH_CHECK();
        }
        k_phi<T, R><<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(psi, w, N, (int)M, nrhs, phi_new);
        JS_LAUNCH_CHECK();
        JS_CUDA(cudaMemsetAsync(acc, 0, 2 * 8 * 8, s));
        k_resid<T><<<dim3(grid_for(N, 256, 152 * 4), nrhs), 256, 0, s>>>(phi_new, phi_old, N, acc);
        JS_LAUNCH_CHECK();
        k_resid_final<<<1, 32, 0, s>>>(acc, nrhs, resid_d);
        JS_LAUNCH_CHECK();
        JS_CUDA(cudaMemcpyAsync(resid_h, resid_d, (nrhs + 1) * 8, cudaMemcpyDeviceToHost, s));
        JS_CUDA(cudaStreamSynchronize(s));
        phi_old = phi_new;
        if (resid_h[nrhs] < tol) {
            conv = true;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    JS_CUDA(cudaMemcpyAsync(phi_out, phi_new, (size_t)nrhs * N * sizeof(T), cudaMemcpyDeviceToDevice, s));
    JS_CUDA(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = resid_h[nrhs];
    if (!conv) {
        set_error("source iteration did not reach tol %g in %d iterations (residual %g)", tol, max_iters,
                  resid_h[nrhs]);
        return JSWEEP_ERR_NOT_CONVERGED;
    }
    return JSWEEP_OK;
}

}  // namespace
}  // namespace js

extern "C" int jsweep_source_iterate_noalloc(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                                             const void *c_ratio, const void *q, const void *inflow, double tol,
                                             int max_iters, void *phi_out, int *iters_out, double *resid_out,
                                             void *stream) {
    using namespace js;
    clear_error();
    if (!dags || !sigma_t || !c_ratio || !q || !phi_out) {
        set_error("jsweep_source_iterate_noalloc: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (nrhs < 1 || nrhs > 8 || (precision != JSWEEP_F64 && precision != JSWEEP_F32)) {
        set_error("jsweep_source_iterate_noalloc: nrhs=%d precision=%d", nrhs, precision);
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (!(tol >= 0.0) || max_iters < 1) {
        set_error("jsweep_source_iterate_noalloc: tol=%g max_iters=%d", tol, max_iters);
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    cudaStream_t s = (cudaStream_t)stream;
    const int Rp = nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8;
#define JS_NA(T, R) si_noalloc_t<T, R>(d, nrhs, sigma_t, c_ratio, q, inflow, tol, max_iters, phi_out, iters_out, resid_out, s)
    if (precision == JSWEEP_F64) {
        switch (Rp) {
            case 1: return JS_NA(double, 1);
            case 2: return JS_NA(double, 2);
            case 4: return JS_NA(double, 4);
            default: return JS_NA(double, 8);
        }
    }
    switch (Rp) {
        case 1: return JS_NA(float, 1);
        case 2: return JS_NA(float, 2);
        case 4: return JS_NA(float, 4);
        default: return JS_NA(float, 8);
    }
#undef JS_NA
}
