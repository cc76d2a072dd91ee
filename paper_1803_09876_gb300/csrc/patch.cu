// Patch programs (JSWEEP_MODE_PATCH): the patch-centric data-driven sweep of
// Sec. V-A / V-B on one GPU.
//
// The cells are grouped into compact patches: a k-d split of pseudo-coordinates
// taken from the levels of the eight octant diagonals (x ~ level(+,+,+) -
// level(-,+,+), ...; the ABI carries no coordinates), or, when the diagonals'
// graphs cannot be built, a recursive breadth-first bisection of the face
// graph.  A program is
// a (patch, octant) pair.  One block runs a program: it stages the patch's
// geometry records and source records in shared memory once, then its warps
// take the octant's directions one after another and sweep each across the
// patch level by level (the entries of a (direction, patch) pair are the
// patch's cells ordered by (level, id)).  Upwind values inside the patch were
// written by the same warp a moment ago; values entering from upwind patches
// are waited for through the per-(cell, direction) epoch flags.
//
// Programs come from a device-wide queue, initially ordered by how far
// upstream the patch lies for the octant.  When a direction's inflow is not
// ready within a short spin, the warp keeps the direction's progress (the
// start of the pass it could not finish: a pass is re-done whole, and the
// values it writes do not change) and moves on; a program with unfinished
// directions goes back to the tail of the queue.  No wait is unbounded, so
// the schedule cannot deadlock however the patches depend on each other; a
// dispatch budget turns a schedule that stops making progress into
// JSWEEP_ERR_DEVICE_TIMEOUT.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "sweep_cell.cuh"

namespace js {

using namespace dev;

// ---- patch partition (host) ----------------------------------------------------------
namespace {

// Recursive bisection: a part larger than the target is split at the median
// breadth-first distance from a pseudo-peripheral cell of the part (found by
// a first breadth-first pass), so parts stay compact.
void bisect_parts(int64_t N, const std::vector<int64_t> &xp, const std::vector<int32_t> &adj, int target,
                  std::vector<int32_t> &cells, std::vector<int32_t> &ptr_out) {
    std::vector<int32_t> tag(N, -1), dist(N, -1), queue;
    queue.reserve(N);
    struct Range { int64_t lo, hi; };
    std::vector<Range> stack{{0, N}};
    std::vector<int32_t> tmp, cnt;
    int32_t next_tag = 0;
    ptr_out.assign(1, 0);
    auto bfs = [&](int32_t src, int32_t t) -> int32_t {  // returns the last cell reached
        queue.clear();
        queue.push_back(src);
        dist[src] = 0;
        size_t h = 0;
        int32_t last = src;
        while (h < queue.size()) {
            const int32_t u = queue[h++];
            last = u;
            for (int64_t e = xp[u]; e < xp[u + 1]; ++e) {
                const int32_t v = adj[e];
                if (tag[v] == t && dist[v] < 0) {
                    dist[v] = dist[u] + 1;
                    queue.push_back(v);
                }
            }
        }
        return last;
    };
    while (!stack.empty()) {
        const Range r = stack.back();
        stack.pop_back();
        const int64_t n = r.hi - r.lo;
        if (n <= target) {
            std::sort(cells.begin() + r.lo, cells.begin() + r.hi);
            ptr_out.push_back((int32_t)r.hi);
            continue;
        }
        const int32_t t = next_tag++;
        for (int64_t i = r.lo; i < r.hi; ++i) {
            tag[cells[i]] = t;
            dist[cells[i]] = -1;
        }
        int32_t far = bfs(cells[r.lo], t);
        for (int64_t i = r.lo; i < r.hi; ++i) dist[cells[i]] = -1;
        bfs(far, t);
        // cells the search did not reach (a disconnected piece) sort last
        int32_t dmax = 0;
        for (int64_t i = r.lo; i < r.hi; ++i) {
            if (dist[cells[i]] < 0) dist[cells[i]] = INT32_MAX;
            else dmax = std::max(dmax, dist[cells[i]]);
        }
        // counting sort by distance (stable: ascending id inside a distance)
        std::sort(cells.begin() + r.lo, cells.begin() + r.hi);
        cnt.assign((size_t)dmax + 2, 0);
        for (int64_t i = r.lo; i < r.hi; ++i) ++cnt[dist[cells[i]] == INT32_MAX ? dmax + 1 : dist[cells[i]]];
        int64_t acc = 0;
        for (auto &x : cnt) {
            const int64_t c = x;
            x = (int32_t)acc;
            acc += c;
        }
        tmp.resize(n);
        for (int64_t i = r.lo; i < r.hi; ++i) {
            const int32_t dd = dist[cells[i]] == INT32_MAX ? dmax + 1 : dist[cells[i]];
            tmp[cnt[dd]++] = cells[i];
        }
        std::copy(tmp.begin(), tmp.end(), cells.begin() + r.lo);
        // split into two parts whose sizes are whole multiples of the target where possible
        const int64_t k = (n + target - 1) / target;
        const int64_t left = std::min<int64_t>(n - 1, std::max<int64_t>(1, (k / 2) * (int64_t)target));
        const int64_t mid = r.lo + (k >= 2 ? left : n / 2);
        stack.push_back({mid, r.hi});  // right half after the left one: patches numbered in traversal order
        stack.push_back({r.lo, mid});
    }
}

// k-d split in pseudo-coordinates: a part larger than the target is cut,
// between two coordinate values, at the median of its widest coordinate, so
// patch interfaces are planes of the coordinate grid.
void kd_parts(const std::vector<int32_t> &x, const std::vector<int32_t> &y, const std::vector<int32_t> &z,
              int target, std::vector<int32_t> &cells, std::vector<int32_t> &ptr_out) {
    struct Range { int64_t lo, hi; };
    std::vector<Range> stack{{0, (int64_t)cells.size()}};
    ptr_out.assign(1, 0);
    const std::vector<int32_t> *co[3] = {&x, &y, &z};
    while (!stack.empty()) {
        const Range r = stack.back();
        stack.pop_back();
        const int64_t n = r.hi - r.lo;
        if (n <= target) {
            std::sort(cells.begin() + r.lo, cells.begin() + r.hi);
            ptr_out.push_back((int32_t)r.hi);
            continue;
        }
        int best = -1;
        int32_t bext = 0;
        for (int a = 0; a < 3; ++a) {
            int32_t lo = INT32_MAX, hi = INT32_MIN;
            for (int64_t i = r.lo; i < r.hi; ++i) {
                lo = std::min(lo, (*co[a])[cells[i]]);
                hi = std::max(hi, (*co[a])[cells[i]]);
            }
            if (hi - lo > bext) {
                bext = hi - lo;
                best = a;
            }
        }
        int64_t mid;
        if (best < 0) {
            mid = r.lo + n / 2;  // all coordinates equal: split by id
            std::sort(cells.begin() + r.lo, cells.begin() + r.hi);
        } else {
            const std::vector<int32_t> &cv = *co[best];
            std::stable_sort(cells.begin() + r.lo, cells.begin() + r.hi,
                             [&](int32_t a, int32_t b) { return cv[a] < cv[b]; });
            // cut between two values, as close to a whole multiple of the target as the ties allow
            const int64_t k = (n + target - 1) / target;
            const int64_t want = r.lo + std::max<int64_t>(1, (k / 2) * (int64_t)target);
            int64_t lo_cut = want, hi_cut = want;
            while (lo_cut > r.lo && cv[cells[lo_cut - 1]] == cv[cells[lo_cut]]) --lo_cut;
            while (hi_cut < r.hi && cv[cells[hi_cut - 1]] == cv[cells[hi_cut]]) ++hi_cut;
            if (lo_cut > r.lo && (want - lo_cut <= hi_cut - want || hi_cut >= r.hi)) mid = lo_cut;
            else if (hi_cut < r.hi) mid = hi_cut;
            else mid = want;  // one value only along this axis (cannot happen: extent > 0)
        }
        stack.push_back({mid, r.hi});
        stack.push_back({r.lo, mid});
    }
}

}  // namespace

int ensure_patch_part(Dags *d, int target, cudaStream_t s) {
    Mesh *mesh = d->mesh;
    if (mesh->part && mesh->part->target == target) return JSWEEP_OK;
    const int64_t N = mesh->N;
    std::vector<int32_t> nb8((size_t)N * 8);
    JS_CUDA(cudaMemcpyAsync(nb8.data(), mesh->nbr8.p, (size_t)N * 32, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> xp(N + 1, 0);
    for (int64_t c = 0; c < N; ++c) {
        int k = 0;
        for (int f = 0; f < 8; ++f) k += nb8[c * 8 + f] >= 0;
        xp[c + 1] = xp[c] + k;
    }
    std::vector<int32_t> adj(xp[N]);
    for (int64_t c = 0; c < N; ++c) {
        int64_t e = xp[c];
        for (int f = 0; f < 8; ++f)
            if (nb8[c * 8 + f] >= 0) adj[e++] = nb8[c * 8 + f];
    }
    std::vector<int32_t> cells(N), ptr;
    std::iota(cells.begin(), cells.end(), 0);
    // pseudo-coordinates from the levels of the octant diagonals: the level for
    // (1,1,1) grows like x + y + z, the one for (-1,1,1) like -x + y + z, ...
    std::unique_ptr<Dags> dg(build_diagonals(d, s));
    std::vector<int32_t> lv;
    if (dg) {
        lv.resize((size_t)8 * N);
        JS_CUDA(cudaMemcpyAsync(lv.data(), dg->level.p, lv.size() * 4, cudaMemcpyDeviceToHost, s));
        JS_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> px(N), py(N), pz(N);
        for (int64_t c = 0; c < N; ++c) {
            const int32_t l0 = lv[c], l1 = lv[1 * N + c], l2 = lv[2 * N + c], l4 = lv[4 * N + c];
            px[c] = l0 - l1;
            py[c] = l0 - l2;
            pz[c] = l0 - l4;
        }
        kd_parts(px, py, pz, target, cells, ptr);
    } else {
        bisect_parts(N, xp, adj, target, cells, ptr);
    }
    const int64_t NP = (int64_t)ptr.size() - 1;
    std::vector<int32_t> pof(N), loc(N);
    int maxP = 0;
    for (int64_t p = 0; p < NP; ++p) {
        maxP = std::max(maxP, ptr[p + 1] - ptr[p]);
        for (int32_t i = ptr[p]; i < ptr[p + 1]; ++i) {
            pof[cells[i]] = (int32_t)p;
            loc[cells[i]] = i - ptr[p];
        }
    }
    // neighbouring patches (undirected), at most kPatchNbrs per patch
    std::vector<int32_t> nbp((size_t)NP * kPatchNbrs, -1);
    for (int64_t p = 0; p < NP; ++p) {
        int32_t *row = nbp.data() + (size_t)p * kPatchNbrs;
        int k = 0;
        for (int32_t i = ptr[p]; i < ptr[p + 1]; ++i) {
            const int32_t c = cells[i];
            for (int64_t e = xp[c]; e < xp[c + 1]; ++e) {
                const int32_t q = pof[adj[e]];
                if (q == (int32_t)p) continue;
                bool seen = false;
                for (int t = 0; t < k; ++t) seen |= row[t] == q;
                if (!seen && k < kPatchNbrs) row[k++] = q;
            }
        }
    }
    auto part = std::make_unique<PatchPart>();
    part->nbp = nbp;
    // dispatch keys: how far downstream a patch lies for each octant diagonal
    part->okey.assign((size_t)8 * NP, -1);
    if (!lv.empty()) {
        for (int o = 0; o < 8; ++o)
            for (int64_t p = 0; p < NP; ++p) {
                int32_t mn = INT32_MAX;
                for (int32_t i = ptr[p]; i < ptr[p + 1]; ++i) mn = std::min(mn, lv[(size_t)o * N + cells[i]]);
                part->okey[(size_t)o * NP + p] = mn;
            }
    }
    JS_TRY(part->d_nbp.alloc(nbp.size() * 4, s));
    JS_CUDA(cudaMemcpyAsync(part->d_nbp.p, nbp.data(), nbp.size() * 4, cudaMemcpyHostToDevice, s));
    part->target = target;
    part->NP = NP;
    part->maxP = maxP;
    part->ptr = ptr;
    JS_TRY(part->d_ptr.alloc((NP + 1) * 4, s));
    JS_TRY(part->d_ids.alloc(N * 4, s));
    JS_TRY(part->d_pof.alloc(N * 4, s));
    JS_TRY(part->d_loc.alloc(N * 4, s));
    JS_CUDA(cudaMemcpyAsync(part->d_ptr.p, ptr.data(), (NP + 1) * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(part->d_ids.p, cells.data(), N * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(part->d_pof.p, pof.data(), N * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(part->d_loc.p, loc.data(), N * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaStreamSynchronize(s));
    mesh->part = std::move(part);
    return JSWEEP_OK;
}

// ---- per-direction patch orders (device) -----------------------------------------------
namespace {

__global__ void k_ps_keys(const int32_t *order, const int32_t *pof, int64_t total, uint32_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)pof[order[i]];
}

// Entry j of direction m: the cell at level-major position perm[m][j], stored as
// its position inside the patch, bit 15 set where a new level of the patch starts.
__global__ void k_ps_entries(const int32_t *order, const int32_t *perm, const uint32_t *skeys, const int32_t *level,
                             const int32_t *loc, const uint8_t *mask, int64_t N, int64_t M, uint16_t *entries,
                             uint8_t *pmask) {
    const int64_t total = N * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N, j = i - m * N;
        const int64_t pos = m * N + perm[i];
        const int32_t c = order[pos];
        const int32_t lev = level[m * N + c];
        bool nl = (j == 0) || skeys[i] != skeys[i - 1];
        if (!nl) {
            const int32_t cp = order[m * N + perm[i - 1]];
            nl = level[m * N + cp] != lev;
        }
        entries[i] = (uint16_t)(loc[c] | (nl ? 0x8000 : 0));
        pmask[i] = mask[pos];
    }
}

// seg[m][p] = first entry of patch p in direction m (keys sorted ascending).
__global__ void k_ps_seg(const uint32_t *skeys, int64_t N, int64_t M, int64_t NP, int32_t *seg) {
    const int64_t total = N * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N, j = i - m * N;
        const uint32_t cur = skeys[i];
        const uint32_t lo = j == 0 ? 0u : skeys[i - 1] + 1;
        if (j == 0 || cur != skeys[i - 1])
            for (uint32_t p = lo; p <= cur; ++p) seg[m * (NP + 1) + p] = (int32_t)j;
        if (j == N - 1)
            for (int64_t p = cur + 1; p <= NP; ++p) seg[m * (NP + 1) + p] = (int32_t)N;
    }
}

// Dispatch key of task (octant o, patch p): the lowest level of the patch's
// cells for the octant's first direction (how far upstream the patch lies).
__global__ void k_ps_task_keys(const int32_t *seg, const int32_t *perm, const int32_t *order, const int32_t *level,
                               const int32_t *oct_dirs, const int32_t *oct_n, int n_oct_max, int64_t N, int64_t NP,
                               int32_t *keys) {
    const int64_t total = 8 * NP;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(t / NP);
        const int64_t p = t - o * NP;
        if (oct_n[o] == 0) {
            keys[t] = -1;
            continue;
        }
        const int m = oct_dirs[o * n_oct_max];
        const int32_t j = seg[m * (NP + 1) + p];
        const int32_t c = order[(int64_t)m * N + perm[(int64_t)m * N + j]];
        keys[t] = level[(int64_t)m * N + c];
    }
}

// Patch dependencies of each octant: bit t of up[o][p] is set when neighbour
// patch nbp[p][t] holds an upwind cell of a cell of p for a direction of octant o
// (entries in level order: order[i] = cell, mask[i] = its incoming faces).
__global__ void k_ps_edges(const int32_t *order, const uint8_t *mask, const int32_t *nbr, const int32_t *pof,
                           const int32_t *nbp, const int32_t *oct_of, int64_t N, int64_t M, int FS, int64_t NP,
                           unsigned long long *up) {
    const int64_t total = N * M;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / N;
        const unsigned msk = mask[i];
        if ((msk & 0x7fu) == 0) continue;
        const int32_t c = order[i];
        const int32_t p = pof[c];
        const int32_t *row = nbp + (int64_t)p * kPatchNbrs;
        unsigned long long bits = 0ull;
        for (int k = 0; k < FS; ++k) {
            if (!((msk >> k) & 1u)) continue;
            const int32_t nb = nbr[(int64_t)c * FS + k];
            if (nb < 0) continue;
            const int32_t q = pof[nb];
            if (q == p) continue;
            for (int t = 0; t < kPatchNbrs && row[t] >= 0; ++t)
                if (row[t] == q) {
                    bits |= 1ull << t;
                    break;
                }
        }
        if (bits) atomicOr(up + (int64_t)oct_of[m] * NP + p, bits);
    }
}

__global__ void k_ps_reset(const int32_t *q_init, int64_t n_ready, int64_t cap, int32_t *queue, uint32_t *seq,
                           uint32_t *ctr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cap; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_ready) queue[i] = q_init[i];
        seq[i] = i < n_ready ? (uint32_t)(i + 1) : 0u;
        if (i == 0) {
            ctr[0] = 0;
            ctr[1] = (uint32_t)n_ready;
            ctr[2] = 0;
            ctr[3] = 0;
            *reinterpret_cast<unsigned long long *>(ctr + 4) = 0ull;
        }
    }
}

}  // namespace

int ensure_patch_sched(Dags *d, cudaStream_t s) {
    const int target = d->opt.patch_cells > 0 ? d->opt.patch_cells : 512;
    if (d->ps && d->ps->target == target) return JSWEEP_OK;
    JS_TRY(ensure_patch_part(d, target, s));
    const PatchPart &pp = *d->mesh->part;
    const int64_t N = d->N, M = d->M, NP = pp.NP;
    if (N * M >= (int64_t)1 << 31) {
        set_error("patch programs: directions x cells must stay below 2^31");
        return JSWEEP_ERR_UNIMPLEMENTED;
    }
    auto ps = std::make_unique<PatchSched>();
    ps->target = target;
    ps->NP = NP;
    // directions of each octant, in increasing index
    std::vector<std::vector<int32_t>> od(8);
    for (int64_t m = 0; m < M; ++m) {
        const double *o = d->quad->dirs.data() + 3 * m;
        od[(o[0] < 0 ? 1 : 0) | (o[1] < 0 ? 2 : 0) | (o[2] < 0 ? 4 : 0)].push_back((int32_t)m);
    }
    int nmax = 1;
    for (auto &v : od) nmax = std::max<int>(nmax, (int)v.size());
    ps->n_oct_max = nmax;
    std::vector<int32_t> odirs((size_t)8 * nmax, 0), on(8);
    int64_t n_tasks = 0;
    for (int o = 0; o < 8; ++o) {
        on[o] = (int32_t)od[o].size();
        for (size_t k = 0; k < od[o].size(); ++k) odirs[(size_t)o * nmax + k] = od[o][k];
        if (on[o] > 0) n_tasks += NP;
    }
    ps->n_tasks = n_tasks;
    ps->cap = 2 * n_tasks;
    int key_bits = 1;
    while ((1ll << key_bits) <= NP) ++key_bits;
    DevBuf keys, skeys, perm;
    JS_TRY(keys.alloc(N * M * 4, s));
    JS_TRY(skeys.alloc(N * M * 4, s));
    JS_TRY(perm.alloc(N * M * 4, s));
    const int32_t *order = d->order.as<int32_t>();  // level-major order of every direction
    k_ps_keys<<<grid_for(N * M, 256, 152 * 64), 256, 0, s>>>(order, pp.d_pof.as<int32_t>(), N * M,
                                                             keys.as<uint32_t>());
    JS_LAUNCH_CHECK();
    // stable: inside a patch the entries keep the (level, id) order
    JS_TRY(radix_sort_segments(keys.as<uint32_t>(), M, N, key_bits, nullptr, perm.as<int32_t>(),
                               skeys.as<uint32_t>(), s));
    JS_TRY(ps->entries.alloc(N * M * 2, s));
    JS_TRY(ps->pmask.alloc(N * M, s));
    JS_TRY(ps->seg.alloc(M * (NP + 1) * 4, s));
    k_ps_entries<<<grid_for(N * M, 256, 152 * 64), 256, 0, s>>>(order, perm.as<int32_t>(), skeys.as<uint32_t>(),
                                                                d->level.as<int32_t>(), pp.d_loc.as<int32_t>(),
                                                                d->mask.as<uint8_t>(), N, M,
                                                                ps->entries.as<uint16_t>(), ps->pmask.as<uint8_t>());
    JS_LAUNCH_CHECK();
    k_ps_seg<<<grid_for(N * M, 256, 152 * 64), 256, 0, s>>>(skeys.as<uint32_t>(), N, M, NP, ps->seg.as<int32_t>());
    JS_LAUNCH_CHECK();
    JS_TRY(ps->oct_dirs.alloc(odirs.size() * 4, s));
    JS_TRY(ps->oct_n.alloc(8 * 4, s));
    JS_CUDA(cudaMemcpyAsync(ps->oct_dirs.p, odirs.data(), odirs.size() * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(ps->oct_n.p, on.data(), 8 * 4, cudaMemcpyHostToDevice, s));
    DevBuf tkeys;
    JS_TRY(tkeys.alloc(8 * NP * 4, s));
    k_ps_task_keys<<<grid_for(8 * NP, 256, 4096), 256, 0, s>>>(ps->seg.as<int32_t>(), perm.as<int32_t>(), order,
                                                               d->level.as<int32_t>(), ps->oct_dirs.as<int32_t>(),
                                                               ps->oct_n.as<int32_t>(), nmax, N, NP,
                                                               tkeys.as<int32_t>());
    JS_LAUNCH_CHECK();
    std::vector<int32_t> tk((size_t)8 * NP);
    JS_CUDA(cudaMemcpyAsync(tk.data(), tkeys.p, tk.size() * 4, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    // prefer the octant diagonal's levels: every direction of the octant crosses
    // a planar patch interface the same way, so they order patches for all of them
    if (!pp.okey.empty() && pp.okey[0] >= 0)
        for (int64_t t = 0; t < 8 * NP; ++t)
            if (tk[t] >= 0) tk[t] = pp.okey[t];
    // rank: upstream patches first, the octants interleaved
    std::vector<int32_t> q;
    q.reserve(n_tasks);
    for (int64_t t = 0; t < 8 * NP; ++t)
        if (tk[t] >= 0) q.push_back((int32_t)t);
    std::stable_sort(q.begin(), q.end(), [&](int32_t a, int32_t b) { return tk[a] < tk[b]; });
    std::vector<int32_t> rank((size_t)8 * NP, -1);
    for (size_t i = 0; i < q.size(); ++i) rank[q[i]] = (int32_t)i;
    // patch dependencies per octant; only the edges that agree with the rank
    // are counted (they form a DAG), the others are left to the yields
    std::vector<int32_t> oof(M);
    for (int o = 0; o < 8; ++o)
        for (int32_t m : od[o]) oof[m] = o;
    DevBuf oof_d, up_d;
    JS_TRY(oof_d.alloc(M * 4, s));
    JS_TRY(up_d.alloc(8 * NP * 8, s));
    JS_CUDA(cudaMemcpyAsync(oof_d.p, oof.data(), M * 4, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemsetAsync(up_d.p, 0, 8 * NP * 8, s));
    k_ps_edges<<<grid_for(N * M, 256, 152 * 64), 256, 0, s>>>(order, d->mask.as<uint8_t>(), d->mesh->nbr.as<int32_t>(),
                                                              pp.d_pof.as<int32_t>(), pp.d_nbp.as<int32_t>(),
                                                              oof_d.as<int32_t>(), N, M, d->mesh->FS, NP,
                                                              up_d.as<unsigned long long>());
    JS_LAUNCH_CHECK();
    std::vector<unsigned long long> up((size_t)8 * NP);
    JS_CUDA(cudaMemcpyAsync(up.data(), up_d.p, up.size() * 8, cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> cnt((size_t)8 * NP, 0), dptr((size_t)8 * NP + 1, 0), dlist;
    std::vector<std::vector<int32_t>> down((size_t)8 * NP);
    for (int32_t t : q) {
        const int o = (int)(t / NP);
        const int64_t p = t - (int64_t)o * NP;
        const unsigned long long bits = up[t];
        for (int b = 0; b < kPatchNbrs; ++b) {
            if (!((bits >> b) & 1ull)) continue;
            const int32_t qn = pp.nbp[(size_t)p * kPatchNbrs + b];
            const int32_t u = (int32_t)(o * NP + qn);
            if (rank[u] >= 0 && rank[u] < rank[t]) {
                ++cnt[t];
                down[u].push_back(t);
            }
        }
    }
    for (size_t t = 0; t < down.size(); ++t) dptr[t + 1] = dptr[t] + (int32_t)down[t].size();
    dlist.reserve(dptr.back());
    for (auto &v : down) dlist.insert(dlist.end(), v.begin(), v.end());
    std::vector<int32_t> ready;
    for (int32_t t : q)
        if (cnt[t] == 0) ready.push_back(t);
    ps->n_ready0 = (int64_t)ready.size();
    if (std::getenv("JSWEEP_VERBOSE")) {
        int64_t fwd = 0, back = 0;
        for (int32_t t : q) {
            const int o = (int)(t / NP);
            const int64_t p = t - (int64_t)o * NP;
            for (int b = 0; b < kPatchNbrs; ++b)
                if ((up[t] >> b) & 1ull) {
                    const int32_t u = (int32_t)(o * NP + pp.nbp[(size_t)p * kPatchNbrs + b]);
                    (rank[u] < rank[t] ? fwd : back) += 1;
                }
        }
        std::fprintf(stderr, "patch programs: %lld patches (largest %d cells), %lld programs, %lld ready, "
                     "%lld forward and %lld backward patch edges\n", (long long)NP, pp.maxP, (long long)n_tasks,
                     (long long)ps->n_ready0, (long long)fwd, (long long)back);
    }
    JS_TRY(ps->q_init.alloc(std::max<size_t>(ready.size(), 1) * 4, s));
    JS_CUDA(cudaMemcpyAsync(ps->q_init.p, ready.data(), ready.size() * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(ps->cnt_init.alloc(cnt.size() * 4, s));
    JS_TRY(ps->cnt.alloc(cnt.size() * 4, s));
    JS_CUDA(cudaMemcpyAsync(ps->cnt_init.p, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(ps->down_ptr.alloc(dptr.size() * 4, s));
    JS_TRY(ps->down.alloc(std::max<size_t>(dlist.size(), 1) * 4, s));
    JS_CUDA(cudaMemcpyAsync(ps->down_ptr.p, dptr.data(), dptr.size() * 4, cudaMemcpyHostToDevice, s));
    if (!dlist.empty())
        JS_CUDA(cudaMemcpyAsync(ps->down.p, dlist.data(), dlist.size() * 4, cudaMemcpyHostToDevice, s));
    JS_TRY(ps->queue.alloc(std::max<int64_t>(ps->cap, 1) * 4, s));
    JS_TRY(ps->seq.alloc(std::max<int64_t>(ps->cap, 1) * 4, s));
    JS_TRY(ps->ctr.alloc(32, s));  // 4 counters, then the watchdog timestamp
    JS_TRY(ps->prog.alloc((size_t)8 * NP * nmax * 4, s));
    JS_CUDA(cudaStreamSynchronize(s));
    d->ps = std::move(ps);
    return JSWEEP_OK;
}

// ---- the patch-program kernel ----------------------------------------------------------
template <class T> struct PatchArgs {
    SweepArgs<T> a;
    const int32_t *pc_ptr, *pc_ids;
    const uint16_t *entries;
    const uint8_t *pmask;
    const int32_t *seg, *oct_dirs, *oct_n;
    int n_oct_max, maxP;
    int64_t NP, n_tasks, cap, dispatch_budget;
    const int32_t *queue;
    int32_t *queue_w;
    uint32_t *seq, *ctr;
    int32_t *prog;
    int *flags;
    int epoch, want;
    int *err;
    long long timeout, yield_cycles, timeout_ns;
    unsigned long long *last_progress;  // %globaltimer of the last finished pass (0 = not started)
    int32_t *cnt;                       // upstream programs still to finish (kForced once queued on demand)
    const int32_t *down_ptr, *down;     // downstream programs
    const int32_t *pof;                 // patch of a cell
};

namespace {

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The per-cell solve of solve_cell (same arithmetic in the same order), with
// the geometry and source records read from shared memory; a wait that is not
// satisfied within yield_cycles returns 1 (the caller yields), an error seen
// on the device returns 2.
template <class T, int R, int SPLIT, int MAXF>
__device__ __forceinline__ int solve_cell_staged(const SweepArgs<T> &a, int m, int c, unsigned msk, int sub,
                                                 const typename V4<T>::type *g, const T *srec, const int *flags,
                                                 int want, const int *err, long long yield_cycles, int &blocker) {
    using V = typename V4<T>::type;
    constexpr int RH = R / SPLIT;
    const T ox = a.dirs[4 * m], oy = a.dirs[4 * m + 1], oz = a.dirs[4 * m + 2];
    V gk[MAXF];
#pragma unroll
    for (int k = 0; k < MAXF; ++k) {
        if (k < a.FS) gk[k] = g[k];
        else gk[k] = V{T(0), T(0), T(0), T(0)};
    }
    T num[RH];
#pragma unroll
    for (int r = 0; r < RH; ++r) num[r] = srec[sub * RH + r];
    T den = srec[R];
    unsigned lagk = 0;
    int lagj[MAXF];
    if (msk & 0x80u) {
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            lagj[k] = -1;
            if (((msk >> k) & 1u) && nbr_bits<T>(gk[k]) >= 0) {
                int j = lag_index(a.lag_ptr, a.lag_face, m, a.sface[(int64_t)c * a.FS + k] >> 1);
                lagj[k] = j;
                if (j >= 0) lagk |= 1u << k;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MAXF; ++k) {
        const int nb = nbr_bits<T>(gk[k]);
        if (((msk >> k) & 1u) && !((lagk >> k) & 1u) && nb >= 0) {
            const int *fp = flags + (int64_t)nb * a.M + m;
            if (ld_acquire(fp) != want) {
                const long long t0 = clock64();
                int ns = 32;
                while (ld_acquire(fp) != want) {
                    if (ld_volatile(err) != 0) return 2;
                    if (clock64() - t0 > yield_cycles) {
                        blocker = nb;
                        return 1;
                    }
                    __nanosleep(ns);
                    ns = ns < 512 ? 2 * ns : 512;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MAXF; ++k) {
        const T d = face_dot(ox, oy, oz, gk[k].x, gk[k].y, gk[k].z);
        if ((msk >> k) & 1u) {
            const T wf = fabs(d);
            const int nb = nbr_bits<T>(gk[k]);
            T up[RH];
            if (nb >= 0) {
                if ((lagk >> k) & 1u) {
                    load_ro<T, RH>(a.psi_lag + (int64_t)lagj[k] * R + sub * RH, up);
                } else {
                    load_cg<T, RH>(a.psi + ((int64_t)nb * a.M + m) * R + sub * RH, up);
                }
            } else {
                const int b = -nb - 1;
#pragma unroll
                for (int r = 0; r < RH; ++r)
                    up[r] = a.inflow ? a.inflow[(int64_t)(sub * RH + r) * a.Fb + b] : T(0);
            }
#pragma unroll
            for (int r = 0; r < RH; ++r) num[r] = fma_rn(wf, up[r], num[r]);
        } else {
            den += d > T(0) ? d : T(0);
        }
    }
    T out[RH];
    const T inv = rcp_rn(den);  // the form every solve uses (sweep_cell.cuh)
#pragma unroll
    for (int r = 0; r < RH; ++r) out[r] = mul_rn(num[r], inv);
    store_cg<T, RH>(a.psi + ((int64_t)c * a.M + m) * R + sub * RH, out);
    return 0;
}

constexpr int kPatchMaxWarps = 12;
constexpr int kWantMax = 32;            // wanted programs recorded per dispatch
constexpr int kForced = INT32_MIN / 2;  // counter of a program queued on demand

template <class T> __device__ __forceinline__ void enqueue_program(const PatchArgs<T> &pa, int task) {
    const uint32_t jq = atomicAdd(pa.ctr + 1, 1u);
    __stcg(pa.queue_w + (int64_t)jq % pa.cap, task);
    __threadfence();
    st_release_u32(pa.seq + (int64_t)jq % pa.cap, jq + 1u);
}

template <class T, int R, int SPLIT, int MAXF>
__global__ void __launch_bounds__(kPatchMaxWarps * 32, 2) k_sweep_patch(const PatchArgs<T> pa) {
    using V = typename V4<T>::type;
    constexpr int RS = src_stride<R>();
    constexpr int CPP = 32 / SPLIT;  // cells per pass
    extern __shared__ __align__(16) unsigned char smem[];
    const int maxP = pa.maxP;
    const int GS = pa.a.GS;
    int32_t *s_ids = reinterpret_cast<int32_t *>(smem);
    V *s_geo = reinterpret_cast<V *>(smem + ((size_t)maxP * 4 + 15) / 16 * 16);
    T *s_src = reinterpret_cast<T *>(s_geo + (size_t)maxP * GS);
    __shared__ int s_task, s_next, s_blocked, s_progress, s_nwant;
    __shared__ int s_want[kWantMax];
    const int lane = threadIdx.x & 31;
    const int cell = lane / SPLIT, sub = lane % SPLIT;
    const SweepArgs<T> &a = pa.a;
    for (;;) {
        if (threadIdx.x == 0) {
            int task = -1;
            const uint32_t i = atomicAdd(pa.ctr + 0, 1u);
            if ((int64_t)i >= pa.dispatch_budget) {
                atomicCAS(pa.err, 0, 3);  // the schedule stopped making progress
            } else {
                const long long t0 = clock64();
                int ns = 64;
                for (;;) {
                    if (ld_acquire_u32(pa.seq + (int64_t)i % pa.cap) == i + 1u) {
                        task = __ldcg(pa.queue + (int64_t)i % pa.cap);
                        break;
                    }
                    if ((int64_t)ld_volatile(reinterpret_cast<const int *>(pa.ctr + 2)) >= pa.n_tasks) break;
                    if (ld_volatile(pa.err) != 0) break;
                    if (clock64() - t0 > pa.timeout) {
                        atomicCAS(pa.err, 0, 2);
                        break;
                    }
                    __nanosleep(ns);
                    ns = ns < 2048 ? 2 * ns : 2048;
                }
                // device-wide watchdog: no pass finished anywhere for longer than the timeout
                if (task >= 0) {
                    const unsigned long long now = globaltimer_ns();
                    unsigned long long lp = __ldcg(pa.last_progress);
                    if (lp == 0ull) {
                        atomicCAS(pa.last_progress, 0ull, now);
                    } else if (now > lp && (long long)(now - lp) > pa.timeout_ns) {
                        atomicCAS(pa.err, 0, 2);
                        task = -1;
                    }
                }
            }
            s_task = task;
            s_next = 0;
            s_blocked = 0;
            s_progress = 0;
            s_nwant = 0;
        }
        __syncthreads();
        const int task = s_task;
        if (task < 0) return;
        const int o = (int)(task / pa.NP);
        const int64_t p = task - (int64_t)o * pa.NP;
        // stage the patch: cell ids, geometry records, source records
        const int c0 = pa.pc_ptr[p], n = pa.pc_ptr[p + 1] - c0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s_ids[i] = pa.pc_ids[c0 + i];
        for (int i = threadIdx.x; i < n * GS; i += blockDim.x) {
            const int q = i / GS;
            s_geo[i] = a.geo[(int64_t)pa.pc_ids[c0 + q] * GS + (i - q * GS)];
        }
        for (int i = threadIdx.x; i < n * RS; i += blockDim.x) {
            const int q = i / RS;
            s_src[i] = a.srcv[(int64_t)pa.pc_ids[c0 + q] * RS + (i - q * RS)];
        }
        __syncthreads();
        const int nd = pa.oct_n[o];
        // warps take the octant's directions; if any yielded, a second round
        // (after a barrier, so no two warps ever hold one direction) retries them
        for (int round = 0; round < 2; ++round) {
            for (;;) {
                int kd = 0;
                if (lane == 0) kd = atomicAdd(&s_next, 1);
                kd = __shfl_sync(0xffffffffu, kd, 0);
                if (kd >= nd) break;
                const int m = pa.oct_dirs[o * pa.n_oct_max + kd];
                int32_t *pg = pa.prog + (int64_t)task * pa.n_oct_max + kd;
                const int seg0 = pa.seg[(int64_t)m * (pa.NP + 1) + p];
                const int seg1 = pa.seg[(int64_t)m * (pa.NP + 1) + p + 1];
                const int j0 = seg0 + __ldcg(pg);
                int j = j0;
                if (j >= seg1) continue;
                bool yielded = false;
                while (j < seg1) {
                    const int jj = j + cell;
                    const uint16_t e = jj < seg1 ? pa.entries[(int64_t)m * a.N + jj] : (uint16_t)0x8000;
                    // a pass ends before the next cell that starts a new level
                    const bool stop = cell > 0 && (e & 0x8000u);
                    const unsigned b = __ballot_sync(0xffffffffu, stop && sub == 0);
                    const int cnt = b ? (__ffs(b) - 1) / SPLIT : CPP;
                    const bool act = cell < cnt && jj < seg1;
                    int st = 0, c = -1, blocker = -1;
                    if (act) {
                        const int l = e & 0x7fff;
                        c = s_ids[l];
                        st = solve_cell_staged<T, R, SPLIT, MAXF>(a, m, c, pa.pmask[(int64_t)m * a.N + jj], sub,
                                                                  s_geo + (size_t)l * GS, s_src + (size_t)l * RS,
                                                                  pa.flags, pa.want, pa.err, pa.yield_cycles,
                                                                  blocker);
                    }
                    const unsigned yl = __ballot_sync(0xffffffffu, st != 0);
                    if (yl) {
                        // the whole pass is re-done later; the program that holds the
                        // first blocking cell is wanted
                        const int bl = __shfl_sync(0xffffffffu, blocker, __ffs(yl) - 1);
                        if (lane == 0 && bl >= 0) {
                            const int w = atomicAdd(&s_nwant, 1);
                            if (w < kWantMax) s_want[w] = o * (int)pa.NP + pa.pof[bl];
                        }
                        yielded = true;
                        break;
                    }
                    if constexpr (SPLIT > 1) {
                        __threadfence();
                        __syncwarp();
                    }
                    if (act && sub == 0) st_release(pa.flags + (int64_t)c * a.M + m, pa.epoch);
                    __syncwarp();
                    j += cnt;
                }
                if (lane == 0) {
                    __stcg(pg, j - seg0);
                    if (yielded) s_blocked = round + 1;
                    if (j > j0) s_progress = 1;
                }
            }
            __syncthreads();
            if (s_blocked != round + 1) break;  // nothing yielded in this round
            __syncthreads();
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            __threadfence();  // progress records before the program is queued again
            if (s_progress) atomicMax(pa.last_progress, globaltimer_ns());
            if (s_blocked == 2) {
                // unfinished: back to the queue; the programs it waits for are
                // queued now if their upstream programs have not all finished
                // (a two-way patch pair would otherwise wait for itself)
                const int nw = min(s_nwant, kWantMax);
                for (int w = 0; w < nw; ++w) {
                    const int wt = s_want[w];
                    if (__ldcg(pa.cnt + wt) > 0 && atomicExch(pa.cnt + wt, kForced) > 0) enqueue_program(pa, wt);
                }
                enqueue_program(pa, task);
                atomicAdd(pa.ctr + 3, 1u);
            } else {
                // finished: queue the downstream programs whose last upstream program this was
                for (int e = pa.down_ptr[task]; e < pa.down_ptr[task + 1]; ++e) {
                    const int dn = pa.down[e];
                    if (atomicSub(pa.cnt + dn, 1) == 1) enqueue_program(pa, dn);
                }
                atomicAdd(pa.ctr + 2, 1u);
            }
        }
        __syncthreads();
    }
}

template <class T, int R, int SPLIT, int MAXF> const void *patch_kernel() {
    return reinterpret_cast<const void *>(k_sweep_patch<T, R, SPLIT, MAXF>);
}

}  // namespace

template <class T, int R> int launch_patch(Dags *d, const SweepArgs<T> &a, cudaStream_t s) {
    constexpr int SPLIT = (int)(sizeof(T) * R / 16) > 1 ? (int)(sizeof(T) * R / 16) : 1;
    constexpr int RS = src_stride<R>();
    JS_TRY(ensure_patch_sched(d, s));
    PatchSched &ps = *d->ps;
    const PatchPart &pp = *d->mesh->part;
    const int GS = a.GS;
    const size_t smem = ((size_t)pp.maxP * 4 + 15) / 16 * 16 + (size_t)pp.maxP * GS * sizeof(typename V4<T>::type) +
                        (size_t)pp.maxP * RS * sizeof(T);
    const void *kern = a.FS <= 4 ? patch_kernel<T, R, SPLIT, 4>()
                     : a.FS <= 6 ? patch_kernel<T, R, SPLIT, 6>()
                                 : patch_kernel<T, R, SPLIT, 7>();
    int dev = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem + 64 > (size_t)smem_max) {
        set_error("patch programs: a %d-cell patch needs %zu bytes of shared memory (at most %d); lower patch_cells",
                  pp.maxP, smem, smem_max);
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // warps per block: the octant's directions split evenly over at most kPatchMaxWarps warps
    const int nd = ps.n_oct_max;
    const int per = (nd + kPatchMaxWarps - 1) / kPatchMaxWarps;
    const int nw = std::max(1, (nd + per - 1) / per);
    int occ = 0;
    JS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nw * 32, smem));
    if (occ < 1) {
        set_error("patch programs: no block fits on an SM (%zu bytes of shared memory)", smem);
        return JSWEEP_ERR_INVALID_ARG;
    }
    const int64_t grid = std::min<int64_t>((int64_t)device_sm_count() * occ, ps.n_tasks);
    // sweep epoch (flags as in the data-driven schedule)
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
    JS_CUDA(cudaMemsetAsync(d->counters.p, 0, 8, s));
    JS_CUDA(cudaMemsetAsync(ps.prog.p, 0, ps.prog.bytes, s));
    JS_CUDA(cudaMemcpyAsync(ps.cnt.p, ps.cnt_init.p, ps.cnt.bytes, cudaMemcpyDeviceToDevice, s));
    k_ps_reset<<<grid_for(ps.cap, 256, 4096), 256, 0, s>>>(ps.q_init.as<int32_t>(), ps.n_ready0, ps.cap,
                                                            ps.queue.as<int32_t>(), ps.seq.as<uint32_t>(),
                                                            ps.ctr.as<uint32_t>());
    JS_LAUNCH_CHECK();
    const int khz = device_clock_khz();
    PatchArgs<T> pa;
    pa.a = a;
    pa.pc_ptr = pp.d_ptr.as<int32_t>();
    pa.pc_ids = pp.d_ids.as<int32_t>();
    pa.entries = ps.entries.as<uint16_t>();
    pa.pmask = ps.pmask.as<uint8_t>();
    pa.seg = ps.seg.as<int32_t>();
    pa.oct_dirs = ps.oct_dirs.as<int32_t>();
    pa.oct_n = ps.oct_n.as<int32_t>();
    pa.n_oct_max = ps.n_oct_max;
    pa.maxP = pp.maxP;
    pa.NP = ps.NP;
    pa.n_tasks = ps.n_tasks;
    pa.cap = ps.cap;
    // a program is dispatched once plus once per yield; a schedule that needs
    // far more dispatches than this is not making progress
    pa.dispatch_budget = std::min<int64_t>((int64_t)ps.n_tasks * 4096 + grid, (int64_t)UINT32_MAX - grid - 1);
    pa.queue = ps.queue.as<int32_t>();
    pa.queue_w = ps.queue.as<int32_t>();
    pa.seq = ps.seq.as<uint32_t>();
    pa.ctr = ps.ctr.as<uint32_t>();
    pa.prog = ps.prog.as<int32_t>();
    pa.flags = d->flags.as<int>();
    pa.epoch = epoch;
    pa.want = d->opt.debug_block_waits ? epoch + 1 : epoch;
    pa.err = reinterpret_cast<int *>(d->counters.p);
    pa.timeout = (long long)(d->opt.spin_timeout_s * (double)khz * 1000.0);
    pa.yield_cycles = (long long)(20e-6 * (double)khz * 1000.0);  // 20 us
    pa.timeout_ns = (long long)(d->opt.spin_timeout_s * 1e9);
    pa.last_progress = reinterpret_cast<unsigned long long *>(ps.ctr.as<uint32_t>() + 4);
    pa.cnt = ps.cnt.as<int32_t>();
    pa.pof = pp.d_pof.as<int32_t>();
    pa.down_ptr = ps.down_ptr.as<int32_t>();
    pa.down = ps.down.as<int32_t>();
    void *args[] = {(void *)&pa};
    JS_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(nw * 32), args, smem, s));
    JS_LAUNCH_CHECK();
    d->timing.sweep_launches = 1;
    return JSWEEP_OK;
}

int patch_counts(Dags *d, cudaStream_t s) {
    uint32_t c[4] = {0, 0, 0, 0};
    if (d->ps) {
        JS_CUDA(cudaMemcpyAsync(c, d->ps->ctr.p, 16, cudaMemcpyDeviceToHost, s));
        JS_CUDA(cudaStreamSynchronize(s));
        d->timing.sweep_programs = d->ps->n_tasks;
    }
    d->timing.sweep_requeues = c[3];
    return JSWEEP_OK;
}

template int launch_patch<float, 1>(Dags *, const SweepArgs<float> &, cudaStream_t);
template int launch_patch<float, 2>(Dags *, const SweepArgs<float> &, cudaStream_t);
template int launch_patch<float, 4>(Dags *, const SweepArgs<float> &, cudaStream_t);
template int launch_patch<float, 8>(Dags *, const SweepArgs<float> &, cudaStream_t);
template int launch_patch<double, 1>(Dags *, const SweepArgs<double> &, cudaStream_t);
template int launch_patch<double, 2>(Dags *, const SweepArgs<double> &, cudaStream_t);
template int launch_patch<double, 4>(Dags *, const SweepArgs<double> &, cudaStream_t);
template int launch_patch<double, 8>(Dags *, const SweepArgs<double> &, cudaStream_t);

}  // namespace js
