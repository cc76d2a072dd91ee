// Device code shared by the single-problem sweeps (sweep.cu) and the batched
// sweeps (batch.cu): the argument block of one problem, cached/uncached vector
// loads, the per-cell upwind solve (from the cell geometry, solve_cell, or
// from a face-coefficient record, solve_cell_coef) and the warp reduction of
// phi.  Every floating-point step that two kernels share is written with
// explicitly rounded operations, so all schedules, batches and right-hand-side
// counts give the same bits.
#pragma once

#include <climits>
#include <cstring>

#include "common.cuh"

namespace js {
namespace dev {

constexpr int kWarpsPerBlock = 8;
// warps per block of the level-synchronous slot kernels: a block's registers
// are released only when its last warp exits, so small blocks recycle warp
// slots sooner (workload 3: 8 warps 46.2 ms, 4 warps 45.4 ms, 2 warps 45.1 ms)
constexpr int kLevelWarps = 2;

template <class T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

template <class T> struct SweepArgs {
    int64_t N;
    int M, FS, GS, Fb;
    const int32_t *order;
    const uint8_t *mask;
    const typename V4<T>::type *geo;
    const T *dirs;  // [M][4] (x, y, z, 0)
    const T *srcv;  // [N][RS]: S V of each rhs at [0, R), sigma_t V at [R]
    const T *inflow;  // [R][Fb] or null
    T *psi;           // [N][M][R]
    T *psi_seq;       // [M][N][R] in each direction's sweep order, or null (see solve_cell_coef)
    const T *psi_lag; // [Tl][R]
    const int32_t *lag_ptr, *lag_face, *sface;
    const int4 *units;
    unsigned long long *bounds_err;  // bounds-checked builds: first bad index (else unused)
};

// Bounds-checked builds (JSWEEP_BOUNDS_CHECK): every gather index of the
// sweeps is checked; the first one out of range is recorded in *bounds_err as
// (check code << 56) | index and its access is skipped.  Codes: 1 cell id,
// 2 upwind cell, 3 boundary face, 4 order position, 5 direction.  In other
// builds JS_IN_RANGE is the constant true and the checks compile away.
__device__ __forceinline__ bool in_range(unsigned long long *w, int64_t i, int64_t n, int code) {
    if (i >= 0 && i < n) return true;
    if (w) atomicCAS(w, 0ull, ((unsigned long long)code << 56) | ((unsigned long long)i & 0xffffffffffffffull));
    return false;
}
#ifdef JSWEEP_BOUNDS_CHECK
#define JS_IN_RANGE(args, i, n, code) ::js::dev::in_range((args).bounds_err, (int64_t)(i), (int64_t)(n), (code))
#else
#define JS_IN_RANGE(args, i, n, code) true
#endif

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

template <class T> __device__ __forceinline__ int nbr_bits(const typename V4<T>::type &g);
template <> __device__ __forceinline__ int nbr_bits<float>(const float4 &g) { return __float_as_int(g.w); }
template <> __device__ __forceinline__ int nbr_bits<double>(const double4 &g) {
    return (int)__double_as_longlong(g.w);
}

// R contiguous values through L2 (bypassing L1: values written by other SMs
// during a persistent sweep must not be served from a stale L1 line).
template <class T, int R> __device__ __forceinline__ void load_cg(const T *p, T (&v)[R]) {
    if constexpr (sizeof(T) * R % 16 == 0) {
        constexpr int n16 = sizeof(T) * R / 16;
#pragma unroll
        for (int i = 0; i < n16; ++i) {
            float4 x = __ldcg(reinterpret_cast<const float4 *>(p) + i);
            memcpy(reinterpret_cast<char *>(v) + 16 * i, &x, 16);
        }
    } else if constexpr (sizeof(T) * R == 8) {
        float2 x = __ldcg(reinterpret_cast<const float2 *>(p));
        memcpy(v, &x, 8);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldcg(p + r);
    }
}

template <class T, int R> __device__ __forceinline__ void load_ro(const T *p, T (&v)[R]) {
    if constexpr (sizeof(T) * R % 16 == 0) {
        constexpr int n16 = sizeof(T) * R / 16;
#pragma unroll
        for (int i = 0; i < n16; ++i) {
            float4 x = __ldg(reinterpret_cast<const float4 *>(p) + i);
            memcpy(reinterpret_cast<char *>(v) + 16 * i, &x, 16);
        }
    } else if constexpr (sizeof(T) * R == 8) {
        float2 x = __ldg(reinterpret_cast<const float2 *>(p));
        memcpy(v, &x, 8);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = __ldg(p + r);
    }
}

template <class T, int R> __device__ __forceinline__ void store_cg(T *p, const T (&v)[R]) {
    if constexpr (sizeof(T) * R % 16 == 0) {
        constexpr int n16 = sizeof(T) * R / 16;
#pragma unroll
        for (int i = 0; i < n16; ++i) {
            float4 x;
            memcpy(&x, reinterpret_cast<const char *>(v) + 16 * i, 16);
            __stcg(reinterpret_cast<float4 *>(p) + i, x);
        }
    } else if constexpr (sizeof(T) * R == 8) {
        float2 x;
        memcpy(&x, v, 8);
        __stcg(reinterpret_cast<float2 *>(p), x);
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r) __stcg(p + r, v[r]);
    }
}

// R contiguous values stored with an L2 eviction policy (16-byte pieces; other
// sizes are plain stores through L2).
template <class T, int R> __device__ __forceinline__ void store_hint(T *p, const T (&v)[R], uint64_t pol) {
    if constexpr (sizeof(T) * R % 16 == 0) {
        constexpr int n16 = sizeof(T) * R / 16;
#pragma unroll
        for (int i = 0; i < n16; ++i) {
            float4 x;
            memcpy(&x, reinterpret_cast<const char *>(v) + 16 * i, 16);
            asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(
                             reinterpret_cast<float4 *>(p) + i),
                         "f"(x.x), "f"(x.y), "f"(x.z), "f"(x.w), "l"(pol)
                         : "memory");
        }
    } else {
        store_cg<T, R>(p, v);
    }
}

// ---- L2 eviction priority of read-once streams ---------------------------------------
// A level-synchronous slot reads its unit, order, mask and face-coefficient
// records once per sweep; they are loaded evict-first so that they leave L2
// to the psi values and source records that other slots read again.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float4 ldg_hint(const float4 *p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int4 ldg_hint(const int4 *p, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int ldg_hint(const int32_t *p, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned ldg_hint(const uint8_t *p, uint64_t pol) {
    unsigned v;
    asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Index of the lagged face f of direction m in the lag list, or -1.
__device__ __forceinline__ int lag_index(const int32_t *lag_ptr, const int32_t *lag_face, int m, int32_t f) {
    int lo = lag_ptr[m], hi = lag_ptr[m + 1];
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (lag_face[mid] < f) lo = mid + 1; else hi = mid;
    }
    return (lo < lag_ptr[m + 1] && lag_face[lo] == f) ? lo : -1;
}

// Source record stride: the R values S V, then sigma_t V, padded so that a
// record is 8, 16, 32 or 64 bytes (FP32) and one DRAM transaction brings both.
template <int R> constexpr int src_stride() { return R >= 4 ? 2 * R : (R == 2 ? 4 : 2); }

// Omega . A of one face, rounded the same way in every kernel (explicit
// round-to-nearest operations, no contraction), so that the per-cell solve and
// the precomputed coefficient stream give bit-identical results.
__device__ __forceinline__ float face_dot(float ox, float oy, float oz, float ax, float ay, float az) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ox, ax), __fmul_rn(oy, ay)), __fmul_rn(oz, az));
}
__device__ __forceinline__ double face_dot(double ox, double oy, double oz, double ax, double ay, double az) {
    return __dadd_rn(__dadd_rn(__dmul_rn(ox, ax), __dmul_rn(oy, ay)), __dmul_rn(oz, az));
}

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
// round-to-nearest sums and differences that the compiler may not fuse with a
// neighbouring product or rearrange
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// psi = num / den as num * (1 / den), both correctly rounded: one reciprocal
// serves every right-hand side of a cell (GB300's FP64 division is costly),
// and every solve uses this same form, so all schedules give the same bits.
__device__ __forceinline__ float rcp_rn(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rcp_rn(double a) { return __drcp_rn(a); }

__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Per-cell geometry and bookkeeping shared by the sweep kernels.
template <class T, int MAXF> struct CellGeo {
    typename V4<T>::type g[MAXF];
};

// One (cell, direction) for RH = R / SPLIT right-hand sides, sub-range `sub`
// (SPLIT lanes cooperate on one cell so that each lane moves 16-byte pieces
// and a 32-byte sector is read by one warp instruction).  MAXF >= faces per
// cell; the face loop is unrolled so that the geometry loads of all faces, and
// then the upwind loads of all incoming faces, are in flight together.
// WAIT: before reading an upwind cell's psi, spin (bounded) until that cell's
// flag for this direction shows the current sweep epoch (data-driven schedule).
// Programmatic dependent launch (level-synchronous slots): a slot kernel lets
// the next slot's kernel start early; that kernel reads everything that does
// not change during a sweep (unit, order, mask, geometry, sources) and waits
// for the previous slots to complete only before it reads upwind psi.
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class T, int R, int SPLIT, int MAXF, bool WAIT, bool PDL = false>
__device__ __forceinline__ bool solve_cell(const SweepArgs<T> &a, int m, int c, unsigned msk, int sub,
                                           const int *flags, int want, int *err, long long timeout) {
    using V = typename V4<T>::type;
    constexpr int RH = R / SPLIT;
    if (!JS_IN_RANGE(a, c, a.N, 1)) return true;  // bounds-checked builds: skip a bad cell id
    const T ox = a.dirs[4 * m], oy = a.dirs[4 * m + 1], oz = a.dirs[4 * m + 2];
    const V *g = a.geo + (int64_t)c * a.GS;
    V gk[MAXF];
#pragma unroll
    for (int k = 0; k < MAXF; ++k) {
        if (k < a.FS) gk[k] = g[k];
        else gk[k] = V{T(0), T(0), T(0), T(0)};
    }
    constexpr int RS = src_stride<R>();
    T num[RH];
    load_ro<T, RH>(a.srcv + (int64_t)c * RS + sub * RH, num);
    T den = __ldg(a.srcv + (int64_t)c * RS + R);
    // lagged faces (rare): bit k set when face slot k takes the previous sweep's value
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
    if constexpr (PDL) pdl_wait_prev();  // upwind values come from earlier slots
    if constexpr (WAIT) {
        // wait until every active interior upwind cell of this direction is done
        // (flags are cell-major, [N][M], like psi: the flags of one cell for
        // the directions of an octant share a sector)
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            const int nb = nbr_bits<T>(gk[k]);
            if (((msk >> k) & 1u) && !((lagk >> k) & 1u) && nb >= 0 && JS_IN_RANGE(a, nb, a.N, 2)) {
                const int *fp = flags + (int64_t)nb * a.M + m;
                if (ld_acquire(fp) != want) {
                    const long long t0 = clock64();
                    int ns = 32;
                    while (ld_acquire(fp) != want) {
                        if (ld_volatile(err) != 0) return false;
                        if (clock64() - t0 > timeout) {
                            atomicCAS(err, 0, 1);
                            return false;
                        }
                        __nanosleep(ns);
                        ns = ns < 1024 ? 2 * ns : 1024;
                    }
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
                } else if (JS_IN_RANGE(a, nb, a.N, 2)) {
                    load_cg<T, RH>(a.psi + ((int64_t)nb * a.M + m) * R + sub * RH, up);
                } else {
#pragma unroll
                    for (int r = 0; r < RH; ++r) up[r] = T(0);
                }
            } else {
                const int b = -nb - 1;
                const bool inb = JS_IN_RANGE(a, b, a.Fb, 3);
#pragma unroll
                for (int r = 0; r < RH; ++r)
                    up[r] = (a.inflow && inb) ? a.inflow[(int64_t)(sub * RH + r) * a.Fb + b] : T(0);
            }
#pragma unroll
            for (int r = 0; r < RH; ++r) num[r] = fma_rn(wf, up[r], num[r]);
        } else {
            den += d > T(0) ? d : T(0);
        }
    }
    T out[RH];
    const T inv = rcp_rn(den);
#pragma unroll
    for (int r = 0; r < RH; ++r) out[r] = mul_rn(num[r], inv);
    store_cg<T, RH>(a.psi + ((int64_t)c * a.M + m) * R + sub * RH, out);
    return true;
}

// ---- precomputed face coefficients (level-synchronous sweeps) ---------------------
// Record of one (direction, position) in the sweep order: Omega.A of every
// face slot (face_dot, T) then the slot's neighbour bits (int32), padded to
// 16 bytes.  The sweep then reads one sequential record per cell-direction
// instead of the cell's scattered geometry record.
template <class T, int MAXF> constexpr int coef_record_bytes() {
    return (MAXF * (int)sizeof(T) + MAXF * 4 + 15) / 16 * 16;
}

// The per-cell solve of solve_cell with the coefficients from the record
// (same operations in the same order, so results are bit-identical).
// `upwind_ready()` is called after every load that does not depend on other
// cells and before the upwind psi reads; it returns false to abandon the cell
// (a bounded wait that gave up).
// SEQ: the record's neighbour entries of interior faces are positions in
// direction m's sweep order, not cell ids; upwind values are read from the
// sweep-order copy psi_seq[m][pos][R], and the result is stored at position
// `idx` (= m N + pos) of that copy as well as in the cell-major psi (with an
// evict-first hint: its next reader is the phi reduction after the sweep).
// A slot's cells then write one contiguous run, and the upwind values come
// from the runs the slots just before wrote, which are still in L2; in the
// cell-major layout each 32-byte piece sits in a 128-byte line whose other
// pieces (the cell's other directions) are written at other times.
// MG: every right-hand side has its own sigma_t (energy groups riding the
// right-hand-side dimension): the record holds sigma_t V of each rhs after
// the S V values, and each rhs has its own denominator, accumulated in the
// same order as the single one, so a group gives the bits of a one-rhs sweep
// with its own sigma_t.
template <class T, int R, int SPLIT, int MAXF, bool SEQ = false, bool MG = false, class Ready>
__device__ __forceinline__ bool solve_cell_coef(const SweepArgs<T> &a, int m, int c, unsigned msk, int sub,
                                                const unsigned char *rec, uint64_t pol_stream,
                                                Ready upwind_ready, int64_t idx = 0) {
    constexpr int RB = coef_record_bytes<T, MAXF>();
    if (!JS_IN_RANGE(a, c, a.N, 1)) return true;  // bounds-checked builds: skip a bad cell id
    T dk[MAXF];
    int nbk[MAXF];
    {
        float4 w[RB / 16];
#pragma unroll
        for (int i = 0; i < RB / 16; ++i) w[i] = ldg_hint(reinterpret_cast<const float4 *>(rec) + i, pol_stream);
        const unsigned char *b = reinterpret_cast<const unsigned char *>(w);
        memcpy(dk, b, MAXF * sizeof(T));
        memcpy(nbk, b + MAXF * sizeof(T), MAXF * 4);
    }
    constexpr int RS = src_stride<R>();
    T num[R / SPLIT], den[MG ? R / SPLIT : 1];
    load_ro<T, R / SPLIT>(a.srcv + (int64_t)c * RS + sub * (R / SPLIT), num);
    if constexpr (MG) load_ro<T, R / SPLIT>(a.srcv + (int64_t)c * RS + R + sub * (R / SPLIT), den);
    else den[0] = __ldg(a.srcv + (int64_t)c * RS + R);
    constexpr int RH = R / SPLIT;
    constexpr int ND = MG ? RH : 1;
    unsigned lagk = 0;
    int lagj[MAXF];
    if (msk & 0x80u) {
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            lagj[k] = -1;
            if (((msk >> k) & 1u) && nbk[k] >= 0) {
                int j = lag_index(a.lag_ptr, a.lag_face, m, a.sface[(int64_t)c * a.FS + k] >> 1);
                lagj[k] = j;
                if (j >= 0) lagk |= 1u << k;
            }
        }
    }
    if (!upwind_ready()) return false;
#pragma unroll
    for (int k = 0; k < MAXF; ++k) {
        const T d = dk[k];
        if ((msk >> k) & 1u) {
            const T wf = fabs(d);
            const int nb = nbk[k];
            T up[RH];
            if (nb >= 0) {
                if ((lagk >> k) & 1u) {
                    load_ro<T, RH>(a.psi_lag + (int64_t)lagj[k] * R + sub * RH, up);
                } else if (JS_IN_RANGE(a, nb, a.N, 2)) {
                    if constexpr (SEQ) load_cg<T, RH>(a.psi_seq + ((int64_t)m * a.N + nb) * R + sub * RH, up);
                    else load_cg<T, RH>(a.psi + ((int64_t)nb * a.M + m) * R + sub * RH, up);
                } else {
#pragma unroll
                    for (int r = 0; r < RH; ++r) up[r] = T(0);
                }
            } else {
                const int b = -nb - 1;
                const bool inb = JS_IN_RANGE(a, b, a.Fb, 3);
#pragma unroll
                for (int r = 0; r < RH; ++r)
                    up[r] = (a.inflow && inb) ? a.inflow[(int64_t)(sub * RH + r) * a.Fb + b] : T(0);
            }
#pragma unroll
            for (int r = 0; r < RH; ++r) num[r] = fma_rn(wf, up[r], num[r]);
        } else {
            const T dp = d > T(0) ? d : T(0);
#pragma unroll
            for (int r = 0; r < ND; ++r) den[r] += dp;
        }
    }
    T out[RH];
    const T inv0 = rcp_rn(den[0]);
#pragma unroll
    for (int r = 0; r < RH; ++r) out[r] = mul_rn(num[r], MG ? rcp_rn(den[r]) : inv0);
    if constexpr (SEQ) {
        store_cg<T, RH>(a.psi_seq + idx * R + sub * RH, out);
        store_hint<T, RH>(a.psi + ((int64_t)c * a.M + m) * R + sub * RH, out, pol_stream);
    } else {
        store_cg<T, RH>(a.psi + ((int64_t)c * a.M + m) * R + sub * RH, out);
    }
    return true;
}


// phi[r][c] = sum_m w_m psi[c][m][r]: one warp per cell reads the cell's
// contiguous [M][R] block (coalesced); lane l sums directions l, l+32, ... in
// increasing order (FP32: Kahan-compensated), then the 32 partial sums are
// combined by a fixed butterfly with error-free two-sums.  The order of every
// operation is fixed, so phi does not depend on the sweep's schedule.
template <class T>
__device__ __forceinline__ void two_sum(T a, T b, T &s, T &e) {
    s = add_rn(a, b);
    const T bb = sub_rn(s, a);
    e = add_rn(sub_rn(a, sub_rn(s, bb)), sub_rn(b, bb));
}

// phi of one cell: lane l sums directions l, l+32, ... of the cell's
// contiguous [M][R] block in increasing order (FP32: Kahan-compensated), then
// the 32 partial sums are combined by a fixed butterfly of error-free
// two-sums.  The order of every operation is fixed, so phi does not depend on
// the sweep's schedule or on which kernel calls this; every lane returns the
// full sum.
template <class T, int R>
__device__ __forceinline__ void phi_warp(const T *blk, const T *w, int M, int lane, T (&out)[R]) {
    T s[R], comp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) s[r] = comp[r] = T(0);
    for (int m = lane; m < M; m += 32) {
        T x[R];
        load_cg<T, R>(blk + (int64_t)m * R, x);
        const T wm = w[m];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            // explicit fused multiply-adds: the compiler may not contract these
            // differently in the kernels that share this reduction
            if constexpr (sizeof(T) == 4) {
                const T y = fma_rn(wm, x[r], -comp[r]);
                const T t = add_rn(s[r], y);
                comp[r] = sub_rn(sub_rn(t, s[r]), y);
                s[r] = t;
            } else {
                s[r] = fma_rn(wm, x[r], s[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        T v = s[r], e = -comp[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, v, off);
            const T oe = __shfl_xor_sync(0xffffffffu, e, off);
            // combine the lower and the upper lane in the same order on both sides
            const bool lower = (lane & off) == 0;
            T ss, ee;
            two_sum(lower ? v : ov, lower ? ov : v, ss, ee);
            v = ss;
            e = add_rn(add_rn(lower ? e : oe, lower ? oe : e), ee);
        }
        out[r] = add_rn(v, e);
    }
}

}  // namespace dev

// Patch programs (patch.cu): one launch of the patch-program sweep.
template <class T, int R> int launch_patch(Dags *d, const dev::SweepArgs<T> &a, cudaStream_t s);
// Programs and re-queued programs of the last patch-program sweep (waits for the stream).
int patch_counts(Dags *d, cudaStream_t s);

}  // namespace js
