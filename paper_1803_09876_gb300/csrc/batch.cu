// Batches: many independent source-iteration problems advanced together.
//
// Sec. V-B keeps every angle of a patch in flight at once; here the same idea
// spans problems.  One iteration of a batch is a handful of launches over all
// active problems, replayed from a CUDA graph:
//   k_emission_batch    source records S V (scattering + fixed source) and sigma_t V
//   k_sweep_level_batch level-synchronous sweep, one launch per merged slot (reading
//                       the handles' face-coefficient streams when they all have one
//                       face-slot count), or
//   k_sweep_dd_batch    data-driven sweep of every (problem, direction), one launch
//   k_lag_update_batch  lagged upwind values for the next sweep (cycle breaking)
//   k_phi_resid_batch   phi = sum_m w_m psi_m and the FP64 residual accumulators
//   k_advance           each problem's convergence test, iteration count, epoch
//   k_deliver_batch     phi of the problems that finished into the callers' arrays
// Each problem owns its workspaces (psi and, for level-synchronous batches, its
// copy in sweep order, epoch flags, source records, lagged values, phi
// ping-pong), so problems that share a mesh and its graphs (one handle) are
// independent.  The per-cell solve and the phi reduction are the
// device functions of the single-problem path, so a problem's results in a
// batch are bit-identical to its results alone.
//
// Merged schedule: the single-problem unit tables (topological per direction,
// grouped by schedule slot) are merged slot by slot, problem-minor, and each
// slot is padded with empty units to a multiple of angles_per_warp A.  A warp
// runs A consecutive units side by side; they then come from one slot, in
// which no unit depends on another, so no lane of a warp ever waits for a
// lane of the same warp.  The deadlock argument of the single-problem kernel
// carries over: the merged order is topological for every problem.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "sweep_cell.cuh"

namespace js {

using namespace dev;

namespace {

// Mutable state of one problem, updated on the device by k_advance.
struct ProbState {
    int active;   // 1 while iterating
    int iters;    // sweeps done
    int old_ix;   // phi buffer holding the last iterate (-1: phi = 0)
    int epoch;    // flag stamp of the next sweep
    int state;    // JSWEEP_PROBLEM_*
    int done_now; // finished in the iteration that just ran (its phi goes to phi_out)
    double resid;  // residual of the last sweep
};
static_assert(sizeof(ProbState) == 32, "ProbState layout");

// Immutable per-problem arguments of the batched kernels.
template <class T> struct ProbArgs {
    SweepArgs<T> a;
    int *flags;  // [N][M] epoch stamps, cell-major like psi
    const unsigned char *coef;  // the handle's face-coefficient stream (level-synchronous), or null
    const T *sig, *cr, *q, *vol, *w;
    T *phi[2];
    T *phi_out;  // the caller's output array
    const int32_t *lag_m, *lag_up;
    int64_t Tl;
    double tol;
    int max_iters, nrhs, dbg, pad;
};

constexpr int kAccPerProb = 16;  // [2 R] u64 residual accumulators (R <= 8)

__device__ __forceinline__ int find_seg(const int64_t *pre, int n, int64_t i) {
    int lo = 0, hi = n;  // largest p in [0, n) with pre[p] <= i
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Data-driven sweep over the merged units of all problems.  Warp g runs the
// A units g*A .. g*A + A - 1 (32 / A lanes each); unit t belongs to problem
// uprob[t].  Units of finished problems and padding units are skipped.
template <class T, int R, int SPLIT, int MAXF, int A>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_sweep_dd_batch(const ProbArgs<T> *__restrict__ P, const ProbState *__restrict__ S, const int4 *units,
                     const int32_t *uprob, int64_t n_units, int *err, long long timeout) {
    const int lane = threadIdx.x & 31;
    constexpr int LPU = 32 / A;  // lanes per unit
    const int a_ix = lane / LPU, ll = lane % LPU, cell = ll / SPLIT, sub = ll % SPLIT;
    const int64_t W = (int64_t)gridDim.x * kWarpsPerBlock;
    const int64_t n_groups = (n_units + A - 1) / A;
    for (int64_t g = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); g < n_groups; g += W) {
        if (__shfl_sync(0xffffffffu, lane == 0 ? ld_volatile(err) : 0, 0) != 0) return;
        const int64_t t = g * A + a_ix;
        bool ok = true;
        int c = -1, p = 0, epoch = 0;
        int4 u = make_int4(0, 0, 0, 0);
        if (t < n_units) {
            u = units[t];
            p = uprob[t];
            if (cell < u.z && S[p].active && JS_IN_RANGE(P[p].a, u.x, P[p].a.M, 5) &&
                JS_IN_RANGE(P[p].a, (int64_t)u.y + cell, P[p].a.N, 4)) {
                const ProbArgs<T> &pp = P[p];
                epoch = S[p].epoch;
                const int64_t idx = (int64_t)u.x * pp.a.N + u.y + cell;
                c = __ldg(pp.a.order + idx);
                if (JS_IN_RANGE(pp.a, c, pp.a.N, 1))
                    ok = solve_cell<T, R, SPLIT, MAXF, true>(pp.a, u.x, c, __ldg(pp.a.mask + idx), sub, pp.flags,
                                                             pp.dbg ? epoch + 1 : epoch, err, timeout);
                else
                    c = -1;  // bounds-checked builds: a bad cell id is neither solved nor released
            }
        }
        if constexpr (SPLIT == 1) {
            if (c >= 0 && ok) st_release(P[p].flags + (int64_t)c * P[p].a.M + u.x, epoch);
        } else {
            // the lanes of a cell publish together (A == 1 when SPLIT > 1)
            __threadfence();
            __syncwarp();
            if (c >= 0 && ok && sub == 0) st_release(P[p].flags + (int64_t)c * P[p].a.M + u.x, epoch);
        }
        if (__any_sync(0xffffffffu, !ok)) return;
    }
}

// Level-synchronous batched sweep: one launch per merged schedule slot; the
// units of a slot are independent, so no waits and no flags.
template <class T, int R, int SPLIT, int MAXF, int A, bool COEF, bool SEQ>
__global__ void __launch_bounds__(kLevelWarps * 32)
    k_sweep_level_batch(const ProbArgs<T> *__restrict__ P, const ProbState *__restrict__ S, const int4 *units,
                        const int32_t *uprob, int64_t u0, int64_t nu) {
    pdl_launch_next();
    const int lane = threadIdx.x & 31;
    constexpr int LPU = 32 / A;
    const int a_ix = lane / LPU, ll = lane % LPU, cell = ll / SPLIT, sub = ll % SPLIT;
    const int64_t t = ((int64_t)blockIdx.x * kLevelWarps + (threadIdx.x >> 5)) * A + a_ix;
    if (t >= nu) return;
    if constexpr (COEF) {
        // every problem has its face stream: sequential coefficient records
        const uint64_t pol_stream = l2_evict_first();
        const int4 u = ldg_hint(units + u0 + t, pol_stream);
        const int p = ldg_hint(uprob + u0 + t, pol_stream);
        if (cell < u.z && S[p].active && JS_IN_RANGE(P[p].a, u.x, P[p].a.M, 5) &&
            JS_IN_RANGE(P[p].a, (int64_t)u.y + cell, P[p].a.N, 4)) {
            const ProbArgs<T> &pp = P[p];
            const int64_t idx = (int64_t)u.x * pp.a.N + u.y + cell;
            solve_cell_coef<T, R, SPLIT, MAXF, SEQ>(pp.a, u.x, ldg_hint(pp.a.order + idx, pol_stream),
                                                    ldg_hint(pp.a.mask + idx, pol_stream), sub,
                                                    pp.coef + idx * coef_record_bytes<T, MAXF>(), pol_stream,
                                                    [] {
                                                        pdl_wait_prev();  // upwind values come from earlier slots
                                                        return true;
                                                    },
                                                    idx);
        }
    } else {
        const int4 u = units[u0 + t];
        const int p = uprob[u0 + t];
        if (cell < u.z && S[p].active && JS_IN_RANGE(P[p].a, u.x, P[p].a.M, 5) &&
            JS_IN_RANGE(P[p].a, (int64_t)u.y + cell, P[p].a.N, 4)) {
            const ProbArgs<T> &pp = P[p];
            const int64_t idx = (int64_t)u.x * pp.a.N + u.y + cell;
            solve_cell<T, R, SPLIT, MAXF, false, true>(pp.a, u.x, __ldg(pp.a.order + idx), __ldg(pp.a.mask + idx),
                                                       sub, nullptr, 0, nullptr, 0);
        }
    }
}

// Source records of every active problem: S V = ((c sigma_t phi_old + q) / 4 pi) V
// for each rhs, then sigma_t V (the records of the single-problem path).
template <class T, int R>
__global__ void k_emission_batch(const ProbArgs<T> *P, const ProbState *S, const int64_t *pre, int np,
                                 int64_t total) {
    constexpr int RS = src_stride<R>();
    const T four_pi = T(4.0 * 3.141592653589793);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_seg(pre, np, i);
        if (!S[p].active) continue;
        const ProbArgs<T> &pp = P[p];
        const int64_t c = i - pre[p], N = pp.a.N;
        const int oi = S[p].old_ix;
        const T *phi = oi >= 0 ? pp.phi[oi] : nullptr;
        const T V = pp.vol[c], sg = pp.sig[c];
        const T cs = pp.cr[c] * sg;
        T out[RS];
#pragma unroll
        for (int r = 0; r < RS; ++r) out[r] = T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r < pp.nrhs) {
                const T ph = phi ? phi[(int64_t)r * N + c] : T(0);
                out[r] = (fma_rn(cs, ph, pp.q[(int64_t)r * N + c]) / four_pi) * V;  // as k_emission
            }
        }
        out[R] = sg * V;
        T *rec = const_cast<T *>(pp.a.srcv) + c * RS;
#pragma unroll
        for (int r = 0; r < RS; ++r) rec[r] = out[r];
    }
}

template <class T, int R>
__global__ void k_lag_update_batch(const ProbArgs<T> *P, const ProbState *S, const int64_t *pre, int np,
                                   int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_seg(pre, np, i);
        if (!S[p].active) continue;
        const ProbArgs<T> &pp = P[p];
        const int64_t j = i - pre[p];
        T v[R];
        load_cg<T, R>(pp.a.psi + ((int64_t)pp.lag_up[j] * pp.a.M + pp.lag_m[j]) * R, v);
        T *dst = const_cast<T *>(pp.a.psi_lag) + j * R;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r] = v[r];
    }
}

__device__ __forceinline__ void flush_max(unsigned long long *acc, int nrhs, const double *dmax, const double *pmax) {
    for (int r = 0; r < nrhs; ++r) {
        atomicMax(acc + 2 * r, (unsigned long long)__double_as_longlong(dmax[r]));
        atomicMax(acc + 2 * r + 1, (unsigned long long)__double_as_longlong(pmax[r]));
    }
}

// phi of every active problem (the warp reduction of the single-problem
// path) and the FP64 residual accumulators max |phi_new - phi_old| and
// max |phi_new| per problem and rhs.  Warp w takes a contiguous chunk of the
// concatenated cells and flushes its maxima when the problem changes.
template <class T, int R>
__global__ void k_phi_resid_batch(const ProbArgs<T> *P, const ProbState *S, const int64_t *pre, int np,
                                  int64_t total, unsigned long long *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t chunk = (total + nw - 1) / nw;
    const int64_t c0 = wid * chunk, c1 = min(total, c0 + chunk);
    int cur = -1, curn = 0;
    double dmax[R], pmax[R];
    for (int64_t i = c0; i < c1; ++i) {
        const int p = find_seg(pre, np, i);
        if (p != cur) {
            if (cur >= 0 && lane == 0) flush_max(acc + (int64_t)cur * kAccPerProb, curn, dmax, pmax);
            cur = p;
            curn = P[p].nrhs;
#pragma unroll
            for (int r = 0; r < R; ++r) dmax[r] = pmax[r] = 0.0;
        }
        if (!S[p].active) continue;
        const ProbArgs<T> &pp = P[p];
        const int64_t c = i - pre[p], N = pp.a.N;
        const int oi = S[p].old_ix;
        T *phi_new = pp.phi[oi >= 0 ? 1 - oi : 0];
        const T *phi_old = oi >= 0 ? pp.phi[oi] : nullptr;
        T v[R];
        phi_warp<T, R>(pp.a.psi + c * pp.a.M * R, pp.w, pp.a.M, lane, v);
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (r < pp.nrhs) {
                    phi_new[(int64_t)r * N + c] = v[r];
                    const double a = (double)v[r];
                    const double b = phi_old ? (double)phi_old[(int64_t)r * N + c] : 0.0;
                    dmax[r] = fmax(dmax[r], fabs(a - b));
                    pmax[r] = fmax(pmax[r], fabs(a));
                }
            }
        }
    }
    if (cur >= 0 && lane == 0 && S[cur].active) flush_max(acc + (int64_t)cur * kAccPerProb, curn, dmax, pmax);
}

// Convergence test of each active problem (the residual of the
// single-problem path: max over rhs of max|phi_new - phi_old| / max|phi_new|),
// then the bookkeeping of the next iteration.
template <class T>
__global__ void k_advance(const ProbArgs<T> *P, ProbState *S, int np, unsigned long long *acc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    ProbState st = S[p];
    unsigned long long *ap = acc + (int64_t)p * kAccPerProb;
    st.done_now = 0;
    if (st.active) {
        double worst = 0.0;
        for (int r = 0; r < P[p].nrhs; ++r) {
            const double d = __longlong_as_double((long long)ap[2 * r]);
            const double m = __longlong_as_double((long long)ap[2 * r + 1]);
            const double v = m > 0.0 ? d / m : (d > 0.0 ? INFINITY : 0.0);
            worst = fmax(worst, v);
        }
        st.iters += 1;
        st.resid = worst;
        st.old_ix = st.old_ix >= 0 ? 1 - st.old_ix : 0;
        st.epoch += 1;
        if (worst < P[p].tol) {
            st.active = 0;
            st.state = JSWEEP_PROBLEM_CONVERGED;
            st.done_now = 1;
        } else if (st.iters >= P[p].max_iters) {
            st.active = 0;
            st.state = JSWEEP_PROBLEM_MAX_ITERS;
            st.done_now = 1;
        }
    }
    S[p] = st;
    for (int k = 0; k < kAccPerProb; ++k) ap[k] = 0ull;
}

// phi of the problems that finished in this iteration into the caller's arrays.
template <class T>
__global__ void k_deliver_batch(const ProbArgs<T> *P, const ProbState *S, const int64_t *pre, int np, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_seg(pre, np, i);
        if (!S[p].done_now) continue;
        const ProbArgs<T> &pp = P[p];
        const int64_t c = i - pre[p], N = pp.a.N;
        const T *src = pp.phi[S[p].old_ix];
        for (int r = 0; r < pp.nrhs; ++r) pp.phi_out[(int64_t)r * N + c] = src[(int64_t)r * N + c];
    }
}

// Merged unit table: unit li of table k (slot t) goes to base[t * K + k] + (li - slot_ptr_k[t]).
__global__ void k_merge_units(const int4 *const *src, const int64_t *uoff, const int64_t *sp, const int64_t *spoff,
                              const int64_t *nslots, const int64_t *base, int K, int64_t total, int4 *dst,
                              int32_t *dprob) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_seg(uoff, K, i);
        const int64_t li = i - uoff[k];
        const int64_t *spk = sp + spoff[k];
        int64_t lo = 0, hi = nslots[k];  // slot: largest t with spk[t] <= li
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (spk[mid] <= li) lo = mid;
            else hi = mid;
        }
        const int64_t d = base[lo * K + k] + (li - spk[lo]);
        dst[d] = src[k][li];
        dprob[d] = k;
    }
}

}  // namespace

// One problem of a batch (host side).
struct BatchProb {
    int64_t id = 0;
    Dags *d = nullptr;
    const void *sig = nullptr, *cr = nullptr, *q = nullptr;
    bool has_inflow = false;
    void *phi_out = nullptr;
    double tol = 0.0;
    int max_iters = 1;
    DevBuf psi, psi_seq, srcv, inflow, psi_lag, phi0, phi1, flags;
    ProbState st{};
    ~BatchProb() { dags_release(d); }
};

struct Batch {
    int prec = JSWEEP_F32, nrhs = 1, Rp = 1;
    jsweep_options opt{};
    std::vector<std::unique_ptr<BatchProb>> probs;  // increasing id
    int64_t next_id = 0;
    // device tables of the problems in `act` (indices into probs)
    std::vector<int> act;
    bool dirty = true;
    DevBuf units, uprob, pargs, pstate, acc, cpre, lpre, err;
    int64_t n_units = 0, ncells = 0, nlags = 0;
    int maxf = 4, apw = 1, mode = JSWEEP_MODE_LEVEL_SYNC;
    bool coef_all = false;  // every problem in the tables has its face stream (and one MAXF)
    bool seq_all = false;   // ... with upwind positions, and its sweep-order copy of psi
    std::vector<int64_t> mslot;  // merged table: slot t is [mslot[t], mslot[t + 1])
    std::vector<int64_t> tab_units;  // units of each problem in the table (by position in act)
    // the captured iteration
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double sweep_ms = 0.0, iter_ms = 0.0;
    int64_t launches = 0;  // kernels this batch launched (graph nodes counted per replay)
    // launch / poll: states of the table's problems copied to pinned host memory
    void *h_state = nullptr;
    size_t h_state_bytes = 0;
    bool pending = false;
    int pending_k = 0;
    cudaEvent_t ev_done = nullptr;
    int64_t sweep_nodes = 0;  // sweep launches in one iteration
    double setup_ms = 0.0;     // host time spent rebuilding tables and capturing graphs
    int64_t rebuilds = 0;
    ~Batch() {
        cudaDeviceSynchronize();
        if (h_state) cudaFreeHost(h_state);
        if (ev_done) cudaEventDestroy(ev_done);
        if (graph) cudaGraphExecDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

template <class T, int R> constexpr int split_for() {
    return (int)(sizeof(T) * R / 16) > 1 ? (int)(sizeof(T) * R / 16) : 1;
}

int pad_rhs_b(int nrhs) { return nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8; }

// Level-synchronous batches with the face stream keep a sweep-order copy of
// each problem's psi (as the single-problem path does).
bool wants_psi_seq(const Batch *b) {
    return b->opt.sweep_mode != JSWEEP_MODE_PERSISTENT && !b->opt.no_face_stream && !b->opt.no_sweep_order_psi;
}

int64_t problem_bytes(const Batch *b, const Dags *d, bool has_inflow) {
    const int64_t es = b->prec == JSWEEP_F64 ? 8 : 4, R = b->Rp, N = d->N, M = d->M;
    const int64_t RS = R >= 4 ? 2 * R : (R == 2 ? 4 : 2);
    int64_t bytes = M * N * R * es + M * N * 4 + N * RS * es + std::max<int64_t>(d->T, 1) * R * es +
                    2 * N * b->nrhs * es;
    if (wants_psi_seq(b)) bytes += M * N * R * es;
    if (has_inflow) bytes += std::max<int64_t>(d->mesh->Fb, 1) * R * es;
    return bytes;
}

// Restart a problem from phi = 0.
int restart(BatchProb &p, cudaStream_t s) {
    p.st.active = 1;
    p.st.iters = 0;
    p.st.old_ix = -1;
    p.st.state = JSWEEP_PROBLEM_ACTIVE;
    p.st.resid = INFINITY;
    if (p.st.epoch <= 0 || p.st.epoch > (1 << 30)) {
        JS_CUDA(cudaMemsetAsync(p.flags.p, 0, p.flags.bytes, s));
        p.st.epoch = 1;
    }
    JS_CUDA(cudaMemsetAsync(p.psi_lag.p, 0, p.psi_lag.bytes, s));
    return JSWEEP_OK;
}

template <class T> ProbArgs<T> prob_args(const Batch *b, BatchProb &p) {
    Dags *d = p.d;
    ProbArgs<T> pa{};
    SweepArgs<T> &a = pa.a;
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
        pa.vol = reinterpret_cast<const T *>(d->mesh->vol32.p);
        pa.w = reinterpret_cast<const T *>(d->quad->w32.p);
    } else {
        a.geo = d->mesh->geo64.as<double4>();
        a.dirs = reinterpret_cast<const T *>(d->dirs4_64.p);
        pa.vol = reinterpret_cast<const T *>(d->mesh->vol64.p);
        pa.w = reinterpret_cast<const T *>(d->quad->w64.p);
    }
    a.srcv = p.srcv.as<T>();
    a.inflow = p.has_inflow ? p.inflow.as<T>() : nullptr;
    a.psi = p.psi.as<T>();
    a.psi_seq = p.psi_seq.p ? p.psi_seq.as<T>() : nullptr;  // used only by the sweep-order level kernel
    a.psi_lag = p.psi_lag.as<T>();
    a.lag_ptr = d->lag_ptr.as<int32_t>();
    a.lag_face = d->lag_face.as<int32_t>();
    a.sface = d->mesh->sface.as<int32_t>();
    a.units = nullptr;
    a.bounds_err = bounds_word();
    pa.flags = p.flags.as<int>();
    pa.sig = static_cast<const T *>(p.sig);
    pa.cr = static_cast<const T *>(p.cr);
    pa.q = static_cast<const T *>(p.q);
    pa.phi[0] = p.phi0.as<T>();
    pa.phi[1] = p.phi1.as<T>();
    pa.phi_out = static_cast<T *>(p.phi_out);
    pa.lag_m = d->lag_m.as<int32_t>();
    pa.lag_up = d->lag_up.as<int32_t>();
    pa.Tl = d->T;
    pa.tol = p.tol;
    pa.max_iters = p.max_iters;
    pa.nrhs = b->nrhs;
    pa.dbg = b->opt.debug_block_waits ? 1 : 0;
    return pa;
}

// Unit table of one handle for the batch's options (the options that shape
// the table are set for the call only).
int handle_units(const Batch *b, Dags *d, int max_cells, cudaStream_t s) {
    const jsweep_options saved = d->opt;
    d->opt.cluster_cells = b->opt.cluster_cells;
    d->opt.unit_order = b->opt.unit_order;
    // patch tasks are a single-problem schedule: batches merge slot-ordered tables
    d->opt.priority = (b->opt.priority == JSWEEP_PRIO_PATCH || b->opt.priority == JSWEEP_PRIO_PATCH_SLBD)
                          ? JSWEEP_PRIO_LEVEL
                          : b->opt.priority;
    d->opt.octant_stagger = b->opt.octant_stagger;
    const int rc = ensure_units(d, JSWEEP_MODE_PERSISTENT, max_cells, s);
    d->opt = saved;
    return rc;
}

// Rebuild the device tables for the problems that are still active.
template <class T, int R> int build_tables(Batch *b, cudaStream_t s) {
    constexpr int SPLIT = split_for<T, R>();
    const int A = SPLIT > 1 ? 1 : std::max(1, b->opt.angles_per_warp);
    const int max_cells = 32 / (SPLIT * A);
    b->act.clear();
    for (int i = 0; i < (int)b->probs.size(); ++i)
        if (b->probs[i]->st.active) b->act.push_back(i);
    const int K = (int)b->act.size();
    b->apw = A;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->n_units = b->ncells = b->nlags = 0;
    if (K == 0) {
        b->dirty = false;
        return JSWEEP_OK;
    }
    int FS = 0;
    std::vector<ProbArgs<T>> P(K);
    std::vector<ProbState> S(K);
    std::vector<int64_t> cpre(K + 1, 0), lpre(K + 1, 0), uoff(K + 1, 0), spoff(K + 1, 0), nsl(K);
    std::vector<const int4 *> src(K);
    std::vector<int64_t> sp_all;
    int64_t nslots = 0;
    for (int k = 0; k < K; ++k) {
        BatchProb &p = *b->probs[b->act[k]];
        Dags *d = p.d;
        if (sizeof(T) == 8) JS_TRY(ensure_dirs64x4(d, d->dirs4_64, s));
        JS_TRY(handle_units(b, d, max_cells, s));
        FS = std::max(FS, d->mesh->FS);
        P[k] = prob_args<T>(b, p);
        S[k] = p.st;
        cpre[k + 1] = cpre[k] + d->N;
        lpre[k + 1] = lpre[k] + d->T;
        uoff[k + 1] = uoff[k] + d->ut.n_units;
        src[k] = d->ut.units.as<int4>();
        const auto &sp = d->ut.slot_ptr;
        nsl[k] = (int64_t)sp.size() - 1;
        nslots = std::max(nslots, nsl[k]);
        spoff[k] = (int64_t)sp_all.size();
        sp_all.insert(sp_all.end(), sp.begin(), sp.end());
    }
    // base[t][k]: slot-major, problem-minor; each slot padded to a multiple of A
    std::vector<int64_t> base((size_t)nslots * K);
    int64_t pos = 0;
    b->mslot.assign(nslots + 1, 0);
    for (int64_t t = 0; t < nslots; ++t) {
        b->mslot[t] = pos;
        for (int k = 0; k < K; ++k) {
            const auto &sp = b->probs[b->act[k]]->d->ut.slot_ptr;
            base[t * K + k] = pos;
            if (t < nsl[k]) pos += sp[t + 1] - sp[t];
        }
        pos = (pos + A - 1) / A * A;
    }
    b->n_units = pos;
    b->mslot[nslots] = pos;
    b->tab_units.assign(K, 0);
    for (int k = 0; k < K; ++k) b->tab_units[k] = uoff[k + 1] - uoff[k];
    b->mode = b->opt.sweep_mode == JSWEEP_MODE_PERSISTENT ? JSWEEP_MODE_PERSISTENT : JSWEEP_MODE_LEVEL_SYNC;
    // level-synchronous batches read the handles' face streams when all have one
    // built for the batch's face slot count (the records' layout depends on it):
    // the streams with upwind positions and the problems' sweep-order psi when
    // every problem has both, else the streams with upwind cell ids
    const int mf = FS <= 4 ? 4 : FS <= 6 ? 6 : 7;
    for (int pass = 0; pass < 2; ++pass) {
        const bool seq = pass == 0;
        b->seq_all = seq;
        b->coef_all = b->mode == JSWEEP_MODE_LEVEL_SYNC && !b->opt.no_face_stream;
        for (int k = 0; k < K && b->coef_all; ++k) {
            BatchProb &pr = *b->probs[b->act[k]];
            Dags *d = pr.d;
            const int dmf = d->mesh->FS <= 4 ? 4 : d->mesh->FS <= 6 ? 6 : 7;
            P[k].coef = (dmf == mf && (!seq || pr.psi_seq.p)) ? ensure_face_stream(d, b->prec, s, seq) : nullptr;
            b->coef_all = P[k].coef != nullptr;
        }
        if (b->coef_all) break;
    }
    if (!b->coef_all) b->seq_all = false;
    for (int k = 0; k < K; ++k) {
        if (!b->coef_all) P[k].coef = nullptr;
        if (!b->seq_all) P[k].a.psi_seq = nullptr;
    }
    b->ncells = cpre[K];
    b->nlags = lpre[K];
    b->maxf = FS <= 4 ? 4 : FS <= 6 ? 6 : 7;
    DevBuf src_d, uoff_d, sp_d, spoff_d, nsl_d, base_d;
    JS_TRY(b->units.ensure((size_t)std::max<int64_t>(pos, 1) * 16, s));
    JS_TRY(b->uprob.ensure((size_t)std::max<int64_t>(pos, 1) * 4, s));
    JS_CUDA(cudaMemsetAsync(b->units.p, 0, (size_t)std::max<int64_t>(pos, 1) * 16, s));
    JS_CUDA(cudaMemsetAsync(b->uprob.p, 0, (size_t)std::max<int64_t>(pos, 1) * 4, s));
    JS_TRY(src_d.alloc(K * sizeof(void *), s));
    JS_TRY(uoff_d.alloc((K + 1) * 8, s));
    JS_TRY(sp_d.alloc(std::max<size_t>(sp_all.size(), 1) * 8, s));
    JS_TRY(spoff_d.alloc((K + 1) * 8, s));
    JS_TRY(nsl_d.alloc(K * 8, s));
    JS_TRY(base_d.alloc(std::max<size_t>(base.size(), 1) * 8, s));
    JS_CUDA(cudaMemcpyAsync(src_d.p, src.data(), K * sizeof(void *), cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(uoff_d.p, uoff.data(), (K + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(sp_d.p, sp_all.data(), sp_all.size() * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(spoff_d.p, spoff.data(), (K + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(nsl_d.p, nsl.data(), K * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(base_d.p, base.data(), base.size() * 8, cudaMemcpyHostToDevice, s));
    if (uoff[K] > 0) {
        k_merge_units<<<grid_for(uoff[K], 256, 152 * 16), 256, 0, s>>>(
            src_d.as<const int4 *>(), uoff_d.as<int64_t>(), sp_d.as<int64_t>(), spoff_d.as<int64_t>(),
            nsl_d.as<int64_t>(), base_d.as<int64_t>(), K, uoff[K], b->units.as<int4>(), b->uprob.as<int32_t>());
        JS_LAUNCH_CHECK();
        b->launches += 1;
    }
    JS_TRY(b->pargs.ensure((size_t)K * sizeof(ProbArgs<T>), s));
    JS_TRY(b->pstate.ensure((size_t)K * sizeof(ProbState), s));
    JS_TRY(b->acc.ensure((size_t)K * kAccPerProb * 8, s));
    JS_TRY(b->cpre.ensure((size_t)(K + 1) * 8, s));
    JS_TRY(b->lpre.ensure((size_t)(K + 1) * 8, s));
    JS_TRY(b->err.ensure(16, s));
    JS_CUDA(cudaMemcpyAsync(b->pargs.p, P.data(), (size_t)K * sizeof(ProbArgs<T>), cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(b->pstate.p, S.data(), (size_t)K * sizeof(ProbState), cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemsetAsync(b->acc.p, 0, (size_t)K * kAccPerProb * 8, s));
    JS_CUDA(cudaMemcpyAsync(b->cpre.p, cpre.data(), (K + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemcpyAsync(b->lpre.p, lpre.data(), (K + 1) * 8, cudaMemcpyHostToDevice, s));
    JS_CUDA(cudaMemsetAsync(b->err.p, 0, 16, s));
    JS_CUDA(cudaStreamSynchronize(s));  // the temporaries above are released on return
    b->dirty = false;
    return JSWEEP_OK;
}

template <class T, int R, int SPLIT, int MAXF, int A> void *dd_kernel() {
    return reinterpret_cast<void *>(k_sweep_dd_batch<T, R, SPLIT, MAXF, A>);
}

template <class T, int R, int SPLIT, int MAXF> void *dd_kernel_a(int A) {
    if constexpr (SPLIT == 1) {
        if (A == 2) return dd_kernel<T, R, SPLIT, MAXF, 2>();
        if (A == 4) return dd_kernel<T, R, SPLIT, MAXF, 4>();
    }
    return dd_kernel<T, R, SPLIT, MAXF, 1>();
}

template <class T, int R, int SPLIT, int MAXF, int A> void *level_kernel(bool coef, bool seq) {
    if (coef && seq) return reinterpret_cast<void *>(k_sweep_level_batch<T, R, SPLIT, MAXF, A, true, true>);
    return coef ? reinterpret_cast<void *>(k_sweep_level_batch<T, R, SPLIT, MAXF, A, true, false>)
                : reinterpret_cast<void *>(k_sweep_level_batch<T, R, SPLIT, MAXF, A, false, false>);
}

template <class T, int R, int SPLIT, int MAXF> void *level_kernel_a(int A, bool coef, bool seq) {
    if constexpr (SPLIT == 1) {
        if (A == 2) return level_kernel<T, R, SPLIT, MAXF, 2>(coef, seq);
        if (A == 4) return level_kernel<T, R, SPLIT, MAXF, 4>(coef, seq);
    }
    return level_kernel<T, R, SPLIT, MAXF, 1>(coef, seq);
}

// Queue one batched iteration on stream cs (captured into the graph).
template <class T, int R> int queue_iteration(Batch *b, cudaStream_t cs) {
    constexpr int SPLIT = split_for<T, R>();
    const int K = (int)b->act.size();
    const ProbArgs<T> *P = b->pargs.as<ProbArgs<T>>();
    ProbState *S = b->pstate.as<ProbState>();
    k_emission_batch<T, R><<<grid_for(b->ncells, 256, 152 * 16), 256, 0, cs>>>(P, S, b->cpre.as<int64_t>(), K,
                                                                               b->ncells);
    if (b->mode == JSWEEP_MODE_LEVEL_SYNC) {
        void *lk = b->maxf == 4 ? level_kernel_a<T, R, SPLIT, 4>(b->apw, b->coef_all, b->seq_all)
                 : b->maxf == 6 ? level_kernel_a<T, R, SPLIT, 6>(b->apw, b->coef_all, b->seq_all)
                                : level_kernel_a<T, R, SPLIT, 7>(b->apw, b->coef_all, b->seq_all);
        const int4 *units = b->units.as<int4>();
        const int32_t *uprob = b->uprob.as<int32_t>();
        JS_CUDA(cudaEventRecordWithFlags(b->ev[0], cs, cudaEventRecordExternal));
        b->sweep_nodes = 0;
        for (size_t t = 0; t + 1 < b->mslot.size(); ++t) {
            int64_t u0 = b->mslot[t], nu = b->mslot[t + 1] - b->mslot[t];
            if (nu <= 0) continue;
            const int64_t warps = (nu + b->apw - 1) / b->apw;
            void *args[] = {(void *)&P, (void *)&S, (void *)&units, (void *)&uprob, (void *)&u0, (void *)&nu};
            // programmatic dependent launch: the next slot starts while this one drains
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)((warps + kLevelWarps - 1) / kLevelWarps));
            cfg.blockDim = dim3(kLevelWarps * 32);
            cfg.stream = cs;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            // the first slot reads the source records the emission kernel just
            // wrote: it keeps a full dependency
            cfg.numAttrs = b->sweep_nodes == 0 ? 0 : 1;
            JS_CUDA(cudaLaunchKernelExC(&cfg, lk, args));
            ++b->sweep_nodes;
        }
        JS_CUDA(cudaEventRecordWithFlags(b->ev[1], cs, cudaEventRecordExternal));
    } else {
    void *kern = b->maxf == 4 ? dd_kernel_a<T, R, SPLIT, 4>(b->apw)
               : b->maxf == 6 ? dd_kernel_a<T, R, SPLIT, 6>(b->apw)
                              : dd_kernel_a<T, R, SPLIT, 7>(b->apw);
    int occ = 0;
    JS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWarpsPerBlock * 32, 0));
    if (occ < 1) occ = 1;
    int64_t grid = (int64_t)device_sm_count() * occ;  // every warp resident
    const int64_t groups = (b->n_units + b->apw - 1) / b->apw;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, (groups + kWarpsPerBlock - 1) / kWarpsPerBlock));
    const int khz = device_clock_khz();
    long long timeout = (long long)(b->opt.spin_timeout_s * (double)khz * 1000.0);
    const int4 *units = b->units.as<int4>();
    const int32_t *uprob = b->uprob.as<int32_t>();
    int64_t nu = b->n_units;
    int *err = b->err.as<int>();
    void *args[] = {(void *)&P, (void *)&S, (void *)&units, (void *)&uprob, (void *)&nu, (void *)&err,
                    (void *)&timeout};
    // external event-record nodes: they time the sweep launch on every replay
    JS_CUDA(cudaEventRecordWithFlags(b->ev[0], cs, cudaEventRecordExternal));
    JS_CUDA(cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kWarpsPerBlock * 32), args, 0, cs));
    JS_CUDA(cudaEventRecordWithFlags(b->ev[1], cs, cudaEventRecordExternal));
    b->sweep_nodes = 1;
    }
    if (b->nlags > 0)
        k_lag_update_batch<T, R><<<grid_for(b->nlags, 256, 152 * 16), 256, 0, cs>>>(P, S, b->lpre.as<int64_t>(), K,
                                                                                    b->nlags);
    k_phi_resid_batch<T, R><<<grid_for(b->ncells * 32, 256, 152 * 16), 256, 0, cs>>>(
        P, S, b->cpre.as<int64_t>(), K, b->ncells, b->acc.as<unsigned long long>());
    k_advance<T><<<(K + 127) / 128, 128, 0, cs>>>(P, S, K, b->acc.as<unsigned long long>());
    k_deliver_batch<T><<<grid_for(b->ncells, 256, 152 * 16), 256, 0, cs>>>(P, S, b->cpre.as<int64_t>(), K,
                                                                           b->ncells);
    return JSWEEP_OK;
}

template <class T, int R> int64_t launches_per_iteration(const Batch *b) {
    return b->sweep_nodes + (b->nlags > 0 ? 5 : 4);
}

// Queue up to n_sweeps iterations of the active problems and the copy of
// their states to pinned host memory; returns without waiting.
template <class T, int R> int launch_t(Batch *b, int n_sweeps, cudaStream_t s) {
    bool any = false;
    for (auto &p : b->probs) any |= p->st.active != 0;
    if (!any) return JSWEEP_OK;
    const auto t0 = std::chrono::steady_clock::now();
    const bool rebuilt = b->dirty || !b->graph;
    if (b->dirty) JS_TRY((build_tables<T, R>(b, s)));
    if (!b->ev[0])
        for (auto &e : b->ev) JS_CUDA(cudaEventCreate(&e));
    if (!b->ev_done) JS_CUDA(cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming));
    if (!b->graph) {
        if (!b->cap) JS_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        JS_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = queue_iteration<T, R>(b, b->cap);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (rc != JSWEEP_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) {
            set_error("batch graph capture failed: %s", cudaGetErrorString(e));
            return JSWEEP_ERR_CUDA;
        }
        const cudaError_t e2 = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            b->graph = nullptr;
            set_error("batch graph instantiate failed: %s", cudaGetErrorString(e2));
            return JSWEEP_ERR_CUDA;
        }
    }
    if (rebuilt) {
        b->setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        ++b->rebuilds;
    }
    const int K = (int)b->act.size();
    const size_t need = (size_t)K * sizeof(ProbState) + 16;
    if (b->h_state_bytes < need) {
        if (b->h_state) cudaFreeHost(b->h_state);
        b->h_state = nullptr;
        b->h_state_bytes = 0;
        JS_CUDA(cudaMallocHost(&b->h_state, need));
        b->h_state_bytes = need;
    }
    for (int i = 0; i < n_sweeps; ++i) {
        if (i == n_sweeps - 1) JS_CUDA(cudaEventRecord(b->ev[2], s));
        JS_CUDA(cudaGraphLaunch(b->graph, s));
        if (i == n_sweeps - 1) JS_CUDA(cudaEventRecord(b->ev[3], s));
        note_launches(launches_per_iteration<T, R>(b));
        b->launches += launches_per_iteration<T, R>(b);
    }
    JS_CUDA(cudaMemcpyAsync(b->h_state, b->pstate.p, (size_t)K * sizeof(ProbState), cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaMemcpyAsync(static_cast<char *>(b->h_state) + (size_t)K * sizeof(ProbState), b->err.p, 4,
                            cudaMemcpyDeviceToHost, s));
    JS_CUDA(cudaEventRecord(b->ev_done, s));
    b->pending = true;
    b->pending_k = K;
    return JSWEEP_OK;
}

// The queued iterations have finished: update the host mirrors.
int finish_launch(Batch *b, int64_t *n_active) {
    b->pending = false;
    const int K = b->pending_k;
    const ProbState *S = static_cast<const ProbState *>(b->h_state);
    int errh = 0;
    std::memcpy(&errh, static_cast<const char *>(b->h_state) + (size_t)K * sizeof(ProbState), 4);
    float ms_sweep = 0.f, ms_iter = 0.f;
    if (cudaEventElapsedTime(&ms_sweep, b->ev[0], b->ev[1]) != cudaSuccess) ms_sweep = 0.f;
    if (cudaEventElapsedTime(&ms_iter, b->ev[2], b->ev[3]) != cudaSuccess) ms_iter = 0.f;
    (void)cudaGetLastError();  // a timing query that failed must not fail a later launch check
    b->sweep_ms = ms_sweep;
    b->iter_ms = ms_iter;
    if (errh) {
        JS_CUDA(cudaMemset(b->err.p, 0, 16));
        set_error("batched sweep: a dependency wait exceeded %.3g s", b->opt.spin_timeout_s);
        return JSWEEP_ERR_DEVICE_TIMEOUT;
    }
    int64_t idle_units = 0;
    for (int k = 0; k < K; ++k) {
        BatchProb &p = *b->probs[b->act[k]];
        p.st = S[k];  // a problem that finished had its phi delivered on the device
        if (!p.st.active) idle_units += b->tab_units[k];
    }
    // finished problems stay in the table (their units are skipped) until they
    // hold half of it; then the next launch rebuilds it from the active ones
    if (2 * idle_units > b->n_units) b->dirty = true;
    if (n_active) {
        int64_t all = 0;
        for (auto &p : b->probs) all += p->st.active != 0;
        *n_active = all;
    }
    return JSWEEP_OK;
}

// Wait for a queued launch, if any, and take its results.
int settle(Batch *b, int64_t *n_active) {
    if (b->pending) {
        JS_CUDA(cudaEventSynchronize(b->ev_done));
        return finish_launch(b, n_active);
    }
    if (n_active) {
        int64_t all = 0;
        for (auto &p : b->probs) all += p->st.active != 0;
        *n_active = all;
    }
    return JSWEEP_OK;
}

#define JS_BATCH_DISPATCH(FN, ...)                                   \
    do {                                                             \
        if (b->prec == JSWEEP_F64) {                                 \
            switch (b->Rp) {                                         \
                case 1: return FN<double, 1>(__VA_ARGS__);           \
                case 2: return FN<double, 2>(__VA_ARGS__);           \
                case 4: return FN<double, 4>(__VA_ARGS__);           \
                default: return FN<double, 8>(__VA_ARGS__);          \
            }                                                        \
        }                                                            \
        switch (b->Rp) {                                             \
            case 1: return FN<float, 1>(__VA_ARGS__);                \
            case 2: return FN<float, 2>(__VA_ARGS__);                \
            case 4: return FN<float, 4>(__VA_ARGS__);                \
            default: return FN<float, 8>(__VA_ARGS__);               \
        }                                                            \
    } while (0)

int launch(Batch *b, int n_sweeps, cudaStream_t s) {
    if (b->pending) {
        set_error("jsweep_batch_launch: the previous launch has not been polled to completion");
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_BATCH_DISPATCH(launch_t, b, n_sweeps, s);
}

int step(Batch *b, int n_sweeps, int64_t *n_active, cudaStream_t s) {
    JS_TRY(settle(b, nullptr));
    JS_TRY(launch(b, n_sweeps, s));
    return settle(b, n_active);
}

int restart_all(Batch *b, cudaStream_t s) {
    for (auto &p : b->probs) JS_TRY(restart(*p, s));
    b->dirty = true;
    return JSWEEP_OK;
}

BatchProb *find_id(Batch *b, int64_t id, size_t *pos = nullptr) {
    auto it = std::lower_bound(b->probs.begin(), b->probs.end(), id,
                               [](const std::unique_ptr<BatchProb> &p, int64_t v) { return p->id < v; });
    if (it == b->probs.end() || (*it)->id != id) return nullptr;
    if (pos) *pos = (size_t)(it - b->probs.begin());
    return it->get();
}

}  // namespace
}  // namespace js

using js::Batch;
using js::BatchProb;

static Batch *bimpl(jsweep_batch_t h) { return reinterpret_cast<Batch *>(h); }

extern "C" {

JSWEEP_API int jsweep_batch_create(int precision, int nrhs, const jsweep_options *opt, jsweep_batch_t *out) {
    js::clear_error();
    if (!out || nrhs < 1 || nrhs > 8 || (precision != JSWEEP_F64 && precision != JSWEEP_F32)) {
        js::set_error("jsweep_batch_create: precision=%d nrhs=%d", precision, nrhs);
        return JSWEEP_ERR_INVALID_ARG;
    }
    auto b = std::make_unique<Batch>();
    JS_TRY(js::check_options(opt, &b->opt));
    b->prec = precision;
    b->nrhs = nrhs;
    b->Rp = js::pad_rhs_b(nrhs);
    *out = reinterpret_cast<jsweep_batch_t>(b.release());
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_problem_bytes(jsweep_batch_t batch, jsweep_dags_t dags, int has_inflow, int64_t *bytes) {
    js::clear_error();
    if (!batch || !dags || !bytes) {
        js::set_error("jsweep_batch_problem_bytes: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *bytes = js::problem_bytes(bimpl(batch), impl(dags), has_inflow != 0);
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_add(jsweep_batch_t batch, jsweep_dags_t dags, const void *sigma_t, const void *c_ratio,
                                const void *q, const void *inflow, void *phi_out, double tol, int max_iters,
                                int64_t *id, void *stream) {
    js::clear_error();
    if (!batch || !dags || !sigma_t || !c_ratio || !q || !phi_out) {
        js::set_error("jsweep_batch_add: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (!(tol >= 0.0) || max_iters < 1 || max_iters >= (1 << 30)) {
        js::set_error("jsweep_batch_add: tol=%g max_iters=%d", tol, max_iters);
        return JSWEEP_ERR_INVALID_ARG;
    }
    Batch *b = bimpl(batch);
    if ((int64_t)b->probs.size() >= JSWEEP_BATCH_MAX_PROBLEMS) {
        js::set_error("jsweep_batch_add: the batch holds %d problems already", JSWEEP_BATCH_MAX_PROBLEMS);
        return JSWEEP_ERR_INVALID_ARG;
    }
    js::Dags *d = impl(dags);
    cudaStream_t s = (cudaStream_t)stream;
    JS_TRY(js::settle(b, nullptr));
    auto p = std::make_unique<BatchProb>();
    const size_t es = b->prec == JSWEEP_F64 ? 8 : 4;
    const int64_t N = d->N, M = d->M, R = b->Rp;
    const int64_t RS = R >= 4 ? 2 * R : (R == 2 ? 4 : 2);
    JS_TRY(p->psi.alloc((size_t)M * N * R * es, s));
    if (js::wants_psi_seq(b)) JS_TRY(p->psi_seq.alloc((size_t)M * N * R * es, s));
    JS_TRY(p->flags.alloc((size_t)M * N * 4, s));
    JS_TRY(p->srcv.alloc((size_t)N * RS * es, s));
    JS_TRY(p->psi_lag.alloc((size_t)std::max<int64_t>(d->T, 1) * R * es, s));
    JS_TRY(p->phi0.alloc((size_t)N * b->nrhs * es, s));
    JS_TRY(p->phi1.alloc((size_t)N * b->nrhs * es, s));
    if (inflow) {
        JS_TRY(p->inflow.alloc((size_t)std::max<int64_t>(d->mesh->Fb, 1) * R * es, s));
        JS_CUDA(cudaMemsetAsync(p->inflow.p, 0, p->inflow.bytes, s));
        JS_CUDA(cudaMemcpyAsync(p->inflow.p, inflow, (size_t)b->nrhs * d->mesh->Fb * es, cudaMemcpyDeviceToDevice, s));
    }
    JS_CUDA(cudaMemsetAsync(p->flags.p, 0, p->flags.bytes, s));
    p->st.epoch = 1;
    JS_TRY(js::restart(*p, s));
    JS_CUDA(cudaStreamSynchronize(s));
    p->d = d;
    d->refs.fetch_add(1);
    p->sig = sigma_t;
    p->cr = c_ratio;
    p->q = q;
    p->has_inflow = inflow != nullptr;
    p->phi_out = phi_out;
    p->tol = tol;
    p->max_iters = max_iters;
    p->id = b->next_id++;
    if (id) *id = p->id;
    b->probs.push_back(std::move(p));
    b->dirty = true;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_step(jsweep_batch_t batch, int n_sweeps, int64_t *n_active, void *stream) {
    js::clear_error();
    if (!batch || n_sweeps < 1) {
        js::set_error("jsweep_batch_step: batch=%p n_sweeps=%d", (void *)batch, n_sweeps);
        return JSWEEP_ERR_INVALID_ARG;
    }
    return js::step(bimpl(batch), n_sweeps, n_active, (cudaStream_t)stream);
}

JSWEEP_API int jsweep_batch_launch(jsweep_batch_t batch, int n_sweeps, void *stream) {
    js::clear_error();
    if (!batch || n_sweeps < 1) {
        js::set_error("jsweep_batch_launch: batch=%p n_sweeps=%d", (void *)batch, n_sweeps);
        return JSWEEP_ERR_INVALID_ARG;
    }
    return js::launch(bimpl(batch), n_sweeps, (cudaStream_t)stream);
}

JSWEEP_API int jsweep_batch_poll(jsweep_batch_t batch, int wait, int *done, int64_t *n_active) {
    js::clear_error();
    if (!batch || !done) {
        js::set_error("jsweep_batch_poll: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Batch *b = bimpl(batch);
    if (b->pending && !wait) {
        const cudaError_t q = cudaEventQuery(b->ev_done);
        if (q == cudaErrorNotReady) {
            (void)cudaGetLastError();
            *done = 0;
            return JSWEEP_OK;
        }
        if (q != cudaSuccess) {
            js::set_error("jsweep_batch_poll: %s", cudaGetErrorString(q));
            return JSWEEP_ERR_CUDA;
        }
    }
    *done = 1;
    return js::settle(b, n_active);
}

JSWEEP_API int jsweep_batch_query(jsweep_batch_t batch, int64_t id, int *state, int *iters, double *resid) {
    js::clear_error();
    BatchProb *p = batch ? js::find_id(bimpl(batch), id) : nullptr;
    if (!p) {
        js::set_error("jsweep_batch_query: no problem with id %lld", (long long)id);
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (state) *state = p->st.state;
    if (iters) *iters = p->st.iters;
    if (resid) *resid = p->st.resid;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_remove(jsweep_batch_t batch, int64_t id) {
    js::clear_error();
    size_t pos = 0;
    Batch *b = batch ? bimpl(batch) : nullptr;
    if (!b || !js::find_id(b, id, &pos)) {
        js::set_error("jsweep_batch_remove: no problem with id %lld", (long long)id);
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_TRY(js::settle(b, nullptr));
    cudaDeviceSynchronize();  // no batched launch may still use its buffers
    b->probs.erase(b->probs.begin() + (ptrdiff_t)pos);
    b->dirty = true;  // the tables refer to problems by position
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_clear(jsweep_batch_t batch) {
    js::clear_error();
    if (!batch) {
        js::set_error("jsweep_batch_clear: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_TRY(js::settle(bimpl(batch), nullptr));
    cudaDeviceSynchronize();
    bimpl(batch)->probs.clear();
    bimpl(batch)->dirty = true;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_size(jsweep_batch_t batch, int64_t *n) {
    js::clear_error();
    if (!batch || !n) {
        js::set_error("jsweep_batch_size: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *n = (int64_t)bimpl(batch)->probs.size();
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_source_iterate(jsweep_batch_t batch, int *iters_out, double *resid_out, void *stream) {
    js::clear_error();
    if (!batch) {
        js::set_error("jsweep_batch_source_iterate: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Batch *b = bimpl(batch);
    cudaStream_t s = (cudaStream_t)stream;
    JS_TRY(js::settle(b, nullptr));
    JS_TRY(js::restart_all(b, s));
    int64_t n_active = (int64_t)b->probs.size();
    while (n_active > 0) JS_TRY(js::step(b, 1, &n_active, s));
    bool all = true;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        const BatchProb &p = *b->probs[i];
        if (iters_out) iters_out[i] = p.st.iters;
        if (resid_out) resid_out[i] = p.st.resid;
        all &= p.st.state == JSWEEP_PROBLEM_CONVERGED;
    }
    if (!all) {
        js::set_error("batch source iteration: a problem stopped at its max_iters");
        return JSWEEP_ERR_NOT_CONVERGED;
    }
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_autotune(jsweep_batch_t batch, void *stream, double *best_ms) {
    js::clear_error();
    if (!batch) {
        js::set_error("jsweep_batch_autotune: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Batch *b = bimpl(batch);
    cudaStream_t s = (cudaStream_t)stream;
    JS_TRY(js::settle(b, nullptr));
    struct Cand {
        int mode, cells, apw, order;
    };
    static const Cand cands[] = {
        {JSWEEP_MODE_LEVEL_SYNC, 32, 1, 1}, {JSWEEP_MODE_LEVEL_SYNC, 32, 1, 0}, {JSWEEP_MODE_LEVEL_SYNC, 16, 2, 1},
        {JSWEEP_MODE_LEVEL_SYNC, 8, 4, 1},  {JSWEEP_MODE_PERSISTENT, 32, 1, 1}, {JSWEEP_MODE_PERSISTENT, 16, 2, 1},
        {JSWEEP_MODE_PERSISTENT, 8, 4, 1},  {JSWEEP_MODE_PERSISTENT, 8, 4, 0}};
    const jsweep_options keep = b->opt;
    double best = INFINITY;
    jsweep_options chosen = keep;
    for (const Cand &c : cands) {
        b->opt = keep;
        b->opt.sweep_mode = c.mode;
        b->opt.cluster_cells = c.cells;
        b->opt.angles_per_warp = c.apw;
        b->opt.unit_order = c.order;
        double t = 0.0;
        for (int rep = 0; rep < 2; ++rep) {  // the first sweep warms the tables and the graph
            int rc = js::restart_all(b, s);
            if (rc == JSWEEP_OK) rc = js::step(b, 1, nullptr, s);
            if (rc != JSWEEP_OK) {
                b->opt = keep;
                js::restart_all(b, s);
                return rc;
            }
            t = b->iter_ms;
        }
        if (t < best) {
            best = t;
            chosen = b->opt;
        }
    }
    b->opt = chosen;
    JS_TRY(js::restart_all(b, s));
    JS_CUDA(cudaStreamSynchronize(s));
    if (best_ms) *best_ms = best;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_stats(jsweep_batch_t batch, double *sweep_ms, double *iteration_ms, int64_t *launches,
                                  double *setup_ms, int64_t *rebuilds) {
    js::clear_error();
    if (!batch) {
        js::set_error("jsweep_batch_stats: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (sweep_ms) *sweep_ms = bimpl(batch)->sweep_ms;
    if (iteration_ms) *iteration_ms = bimpl(batch)->iter_ms;
    if (launches) *launches = bimpl(batch)->launches;
    if (setup_ms) *setup_ms = bimpl(batch)->setup_ms;
    if (rebuilds) *rebuilds = bimpl(batch)->rebuilds;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_options(jsweep_batch_t batch, jsweep_options *out) {
    js::clear_error();
    if (!batch || !out) {
        js::set_error("jsweep_batch_options: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *out = bimpl(batch)->opt;
    return JSWEEP_OK;
}

JSWEEP_API int jsweep_batch_destroy(jsweep_batch_t batch) {
    delete bimpl(batch);
    return JSWEEP_OK;
}

}  // extern "C"
