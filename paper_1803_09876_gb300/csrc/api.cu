#include <algorithm>
// C ABI entry points: errors, allocator, mesh and quadrature handles, option
// handling and the dependency-graph handle's host-side accessors.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include <atomic>

#include "common.cuh"

namespace js {

std::atomic<int64_t> g_kernel_launches{0};

// ---- errors ---------------------------------------------------------------------
static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

// ---- allocator ------------------------------------------------------------------
static std::mutex g_alloc_mu;
static jsweep_alloc_fn g_alloc = nullptr;
static jsweep_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

int DevBuf::alloc(size_t nbytes, cudaStream_t s) {
    release();
    if (nbytes == 0) return JSWEEP_OK;
    jsweep_alloc_fn a;
    jsweep_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc; f = g_free; ctx = g_alloc_ctx;
    }
    size_t rounded = (nbytes + 255) & ~size_t(255);
    if (a) {
        p = a(rounded, (void *)s, ctx);
        if (!p) {
            set_error("device allocation of %zu bytes failed (user allocator)", rounded);
            return JSWEEP_ERR_OOM;
        }
        free_fn = f;
        free_ctx = ctx;
    } else {
        cudaError_t e = cudaMalloc(&p, rounded);
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            set_error("cudaMalloc of %zu bytes failed: %s", rounded, cudaGetErrorString(e));
            return JSWEEP_ERR_OOM;
        }
        free_fn = nullptr;
    }
    bytes = rounded;
    return JSWEEP_OK;
}

int DevBuf::ensure(size_t nbytes, cudaStream_t s) {
    if (p && bytes >= nbytes) return JSWEEP_OK;
    return alloc(nbytes, s);
}

void DevBuf::release() {
    if (!p) return;
    if (free_fn) {
        free_fn(p, bytes, nullptr, free_ctx);
    } else {
        cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
    free_fn = nullptr;
}

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

// Error word of the bounds-checked build on the current device (8 bytes, zeroed,
// allocated once per device and kept for the process); nullptr in other builds.
unsigned long long *bounds_word() {
#ifdef JSWEEP_BOUNDS_CHECK
    static std::mutex mu;
    static unsigned long long *words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!words[dev]) {
        void *p = nullptr;
        if (cudaMalloc(&p, 8) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        cudaMemset(p, 0, 8);
        words[dev] = static_cast<unsigned long long *>(p);
    }
    return words[dev];
#else
    return nullptr;
#endif
}

// SM clock (kHz) of the current device, queried once per device: the query is
// slow enough to show between the events of a short sweep.
int device_clock_khz() {
    static std::atomic<int> cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 2000000;
    int khz = dev < 64 ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (khz > 0) return khz;
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2000000;
    if (dev < 64) cache[dev].store(khz, std::memory_order_relaxed);
    return khz;
}

void mesh_release(Mesh *m) {
    if (m && m->refs.fetch_sub(1) == 1) delete m;
}
void quad_release(Quad *q) {
    if (q && q->refs.fetch_sub(1) == 1) delete q;
}
void dags_release(Dags *d) {
    if (d && d->refs.fetch_sub(1) == 1) {
        cudaDeviceSynchronize();
        delete d;
    }
}

Dags::~Dags() {
    if (graph) cudaGraphExecDestroy(graph);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    mesh_release(mesh);
    quad_release(quad);
}

// ---- Gauss-Legendre nodes by Newton's method on the three-term recurrence ------
// (P_0 = 1, P_1 = x, (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};
//  P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weight 2 / ((1 - x^2) P_n'(x)^2)).
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            // p1 = P_n(z), p0 = P_{n-1}(z)
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-17) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        // nodes ascending: x[n-1-i] = z (positive side), x[i] = -z
        x[n - 1 - i] = z;
        x[i] = -z;
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        w[n - 1 - i] = wi;
        w[i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

}  // namespace js

using namespace js;

extern "C" {

const char *jsweep_last_error(void) { return g_err; }

int jsweep_version(void) { return 100; }

int jsweep_options_default(jsweep_options *opt) {
    if (!opt) {
        set_error("jsweep_options_default: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    std::memset(opt, 0, sizeof(*opt));
    opt->struct_size = (int)sizeof(jsweep_options);
    opt->sweep_mode = JSWEEP_MODE_AUTO;
    opt->priority = JSWEEP_PRIO_LEVEL;
    opt->cluster_cells = 32;
    opt->blocks_per_sm = 0;
    opt->octant_stagger = 0;
    opt->spin_timeout_s = 2.0;
    opt->cycle_search_max = 256;
    opt->unit_order = 1;
    opt->angles_per_warp = 1;
    opt->patch_cells = 512;
    opt->eager_search_max = 64;
    return JSWEEP_OK;
}

int jsweep_set_allocator(jsweep_alloc_fn alloc, jsweep_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("jsweep_set_allocator: give both functions or neither");
        return JSWEEP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = ctx;
    return JSWEEP_OK;
}

// ---- mesh ---------------------------------------------------------------------------
int jsweep_mesh_create(int64_t n_cells, int64_t n_faces, const int64_t *face_cells,
                       const double *normals, const double *areas, const double *volumes,
                       jsweep_mesh_t *out) {
    clear_error();
    if (!out || !face_cells || !normals || !areas || !volumes) {
        set_error("jsweep_mesh_create: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n_cells <= 0 || n_faces <= 0 || n_cells >= INT32_MAX || n_faces >= INT32_MAX / 2) {
        set_error("jsweep_mesh_create: n_cells=%lld n_faces=%lld out of range",
                  (long long)n_cells, (long long)n_faces);
        return JSWEEP_ERR_INVALID_ARG;
    }
    const int64_t N = n_cells, F = n_faces;
    std::vector<int> nf(N, 0);
    std::vector<double> net(3 * N, 0.0), asum(N, 0.0);
    int64_t Fb = 0;
    for (int64_t f = 0; f < F; ++f) {
        int64_t c0 = face_cells[2 * f], c1 = face_cells[2 * f + 1];
        if (c0 < 0 || c0 >= N || c1 < -1 || c1 >= N || c1 == c0) {
            set_error("mesh invalid: face %lld has cells (%lld, %lld)", (long long)f,
                      (long long)c0, (long long)c1);
            return JSWEEP_ERR_MESH_INVALID;
        }
        double a = areas[f];
        const double *n = normals + 3 * f;
        double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(a > 0.0) || !std::isfinite(a)) {
            set_error("mesh invalid: face %lld has area %g", (long long)f, a);
            return JSWEEP_ERR_MESH_INVALID;
        }
        if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6) {
            set_error("mesh invalid: face %lld normal is not a unit vector (|n| = %g)",
                      (long long)f, nn);
            return JSWEEP_ERR_MESH_INVALID;
        }
        nf[c0]++;
        asum[c0] += a;
        for (int k = 0; k < 3; ++k) net[3 * c0 + k] += a * n[k];
        if (c1 >= 0) {
            nf[c1]++;
            asum[c1] += a;
            for (int k = 0; k < 3; ++k) net[3 * c1 + k] -= a * n[k];
        } else {
            ++Fb;
        }
    }
    int FS = 0;
    for (int64_t c = 0; c < N; ++c) {
        double v = volumes[c];
        if (!(v > 0.0) || !std::isfinite(v)) {
            set_error("mesh invalid: cell %lld has volume %g", (long long)c, v);
            return JSWEEP_ERR_MESH_INVALID;
        }
        if (nf[c] == 0 || nf[c] > kMaxFaces) {
            set_error("mesh invalid: cell %lld has %d faces (1..%d supported)", (long long)c,
                      nf[c], kMaxFaces);
            return nf[c] == 0 ? JSWEEP_ERR_MESH_INVALID : JSWEEP_ERR_UNIMPLEMENTED;
        }
        double r = std::sqrt(net[3 * c] * net[3 * c] + net[3 * c + 1] * net[3 * c + 1] +
                             net[3 * c + 2] * net[3 * c + 2]);
        if (r > 1e-8 * asum[c]) {
            set_error("mesh invalid: cell %lld is not closed (|sum a n| = %g, sum a = %g)",
                      (long long)c, r, asum[c]);
            return JSWEEP_ERR_MESH_INVALID;
        }
        if (nf[c] > FS) FS = nf[c];
    }
    // slots per cell, faces in increasing id
    // geometry records padded to 4 or 8 slots: a hexahedron's record is one 128-byte line (FP32)
    const int GS = FS <= 4 ? 4 : 8;
    std::vector<int32_t> sface(N * FS, -1), nbr(N * FS, INT32_MIN);
    std::vector<float> geo32(N * GS * 4, 0.0f);
    std::vector<double> geo64(N * GS * 4, 0.0);
    std::vector<int> fill(N, 0);
    int64_t b = 0;
    for (int64_t f = 0; f < F; ++f) {
        int64_t c0 = face_cells[2 * f], c1 = face_cells[2 * f + 1];
        int32_t bid = -1;
        if (c1 < 0) bid = (int32_t)(b++);
        for (int side = 0; side < 2; ++side) {
            int64_t c = side == 0 ? c0 : c1;
            if (c < 0) continue;
            int k = fill[c]++;
            int64_t slot = c * FS + k;
            int64_t gslot = c * GS + k;
            sface[slot] = (int32_t)((f << 1) | side);
            int32_t nb = side == 0 ? (c1 >= 0 ? (int32_t)c1 : -(bid + 1)) : (int32_t)c0;
            nbr[slot] = nb;
            double sg = side == 0 ? 1.0 : -1.0;
            for (int k3 = 0; k3 < 3; ++k3) {
                double av = sg * areas[f] * normals[3 * f + k3];
                geo64[4 * gslot + k3] = av;
                geo32[4 * gslot + k3] = (float)av;
            }
            int32_t nb32 = nb;
            std::memcpy(&geo32[4 * gslot + 3], &nb32, 4);
            long long nb64 = nb;
            std::memcpy(&geo64[4 * gslot + 3], &nb64, 8);
        }
    }
    for (int64_t c = 0; c < N; ++c) {
        for (int k = fill[c]; k < GS; ++k) {  // empty slots: zero area, marker neighbour
            int64_t gslot = c * GS + k;
            int32_t nb32 = INT32_MIN;
            std::memcpy(&geo32[4 * gslot + 3], &nb32, 4);
            long long nb64 = INT32_MIN;
            std::memcpy(&geo64[4 * gslot + 3], &nb64, 8);
        }
    }
    std::vector<float> vol32(N);
    for (int64_t c = 0; c < N; ++c) vol32[c] = (float)volumes[c];

    Mesh *m = new Mesh();
    m->N = N;
    m->F = F;
    m->Fb = Fb;
    m->FS = FS;
    m->GS = GS;
    cudaStream_t s = nullptr;
    int rc = JSWEEP_OK;
    auto up = [&](DevBuf &buf, const void *src, size_t bytes) {
        if (rc != JSWEEP_OK) return;
        rc = buf.alloc(bytes, s);
        if (rc != JSWEEP_OK) return;
        cudaError_t e = cudaMemcpy(buf.p, src, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            set_error("cudaMemcpy: %s", cudaGetErrorString(e));
            rc = JSWEEP_ERR_CUDA;
        }
    };
    up(m->sface, sface.data(), sface.size() * 4);
    up(m->nbr, nbr.data(), nbr.size() * 4);
    {
        std::vector<int32_t> nbr8(N * 8, INT32_MIN);
        for (int64_t c = 0; c < N; ++c)
            for (int k = 0; k < FS; ++k) nbr8[c * 8 + k] = nbr[c * FS + k];
        up(m->nbr8, nbr8.data(), nbr8.size() * 4);
    }
    up(m->normal, normals, F * 3 * sizeof(double));
    up(m->geo32, geo32.data(), geo32.size() * 4);
    up(m->geo64, geo64.data(), geo64.size() * 8);
    up(m->vol64, volumes, N * 8);
    up(m->vol32, vol32.data(), N * 4);
    if (rc != JSWEEP_OK) {
        delete m;
        return rc;
    }
    *out = reinterpret_cast<jsweep_mesh_t>(m);
    return JSWEEP_OK;
}

int jsweep_mesh_destroy(jsweep_mesh_t mesh) {
    mesh_release(impl(mesh));
    return JSWEEP_OK;
}

int jsweep_mesh_info(jsweep_mesh_t mesh, int64_t *n_cells, int64_t *n_faces, int64_t *n_bfaces,
                     int *max_faces_per_cell) {
    if (!mesh) {
        set_error("jsweep_mesh_info: NULL mesh");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Mesh *m = impl(mesh);
    if (n_cells) *n_cells = m->N;
    if (n_faces) *n_faces = m->F;
    if (n_bfaces) *n_bfaces = m->Fb;
    if (max_faces_per_cell) *max_faces_per_cell = m->FS;
    return JSWEEP_OK;
}

// ---- quadrature ------------------------------------------------------------------------
int jsweep_quadrature_product(int n_polar, int n_azim, double *dirs, double *weights) {
    clear_error();
    if (n_polar < 1 || n_polar > 64 || n_azim < 1 || n_azim > 64 || !dirs || !weights) {
        set_error("jsweep_quadrature_product: n_polar=%d n_azim=%d", n_polar, n_azim);
        return JSWEEP_ERR_INVALID_ARG;
    }
    std::vector<double> x, w;
    gauss_legendre(2 * n_polar, x, w);
    const double pi = 3.14159265358979323846;
    const double wphi = 0.5 * pi / n_azim;
    for (int oct = 0; oct < 8; ++oct) {
        double sx = (oct & 1) ? -1.0 : 1.0, sy = (oct & 2) ? -1.0 : 1.0, sz = (oct & 4) ? -1.0 : 1.0;
        for (int i = 0; i < n_polar; ++i) {
            double mu = x[n_polar + i];
            double st = std::sqrt(1.0 - mu * mu);
            for (int j = 0; j < n_azim; ++j) {
                double ph = (j + 0.5) * (0.5 * pi) / n_azim;
                int64_t m = (int64_t)oct * n_polar * n_azim + (int64_t)i * n_azim + j;
                dirs[3 * m + 0] = sx * st * std::cos(ph);
                dirs[3 * m + 1] = sy * st * std::sin(ph);
                dirs[3 * m + 2] = sz * mu;
                weights[m] = w[n_polar + i] * wphi;
            }
        }
    }
    return JSWEEP_OK;
}

int jsweep_quadrature_create(int64_t n_dirs, const double *dirs, const double *weights,
                             jsweep_quad_t *out) {
    clear_error();
    if (!out || !dirs || !weights || n_dirs <= 0 || n_dirs > 65536) {
        set_error("jsweep_quadrature_create: bad arguments (n_dirs=%lld)", (long long)n_dirs);
        return JSWEEP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int64_t m = 0; m < n_dirs; ++m) {
        const double *o = dirs + 3 * m;
        double nn = o[0] * o[0] + o[1] * o[1] + o[2] * o[2];
        if (!std::isfinite(nn) || nn == 0.0 || !std::isfinite(weights[m])) {
            set_error("jsweep_quadrature_create: direction %lld is zero or not finite", (long long)m);
            return JSWEEP_ERR_INVALID_ARG;
        }
    }
    Quad *q = new Quad();
    q->M = n_dirs;
    q->dirs.assign(dirs, dirs + 3 * n_dirs);
    q->w.assign(weights, weights + n_dirs);
    std::vector<float> d32(4 * n_dirs), w32(n_dirs);
    for (int64_t m = 0; m < n_dirs; ++m) {
        for (int k = 0; k < 3; ++k) d32[4 * m + k] = (float)dirs[3 * m + k];
        d32[4 * m + 3] = 0.0f;
        w32[m] = (float)weights[m];
    }
    int rc = JSWEEP_OK;
    auto up = [&](DevBuf &buf, const void *src, size_t bytes) {
        if (rc != JSWEEP_OK) return;
        rc = buf.alloc(bytes, nullptr);
        if (rc != JSWEEP_OK) return;
        if (cudaMemcpy(buf.p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("cudaMemcpy failed");
            rc = JSWEEP_ERR_CUDA;
        }
    };
    up(q->dirs64, dirs, 3 * n_dirs * 8);
    up(q->dirs32, d32.data(), 4 * n_dirs * 4);
    up(q->w64, weights, n_dirs * 8);
    up(q->w32, w32.data(), n_dirs * 4);
    if (rc != JSWEEP_OK) {
        delete q;
        return rc;
    }
    *out = reinterpret_cast<jsweep_quad_t>(q);
    return JSWEEP_OK;
}

int jsweep_quadrature_destroy(jsweep_quad_t quad) {
    quad_release(impl(quad));
    return JSWEEP_OK;
}

// ---- dependency graphs --------------------------------------------------------------
}  // extern "C"

namespace js {
// Validated copy of the caller's options (defaults where unset).
int check_options(const jsweep_options *opt, jsweep_options *o) {
    jsweep_options_default(o);
    if (!opt) return JSWEEP_OK;
    if (opt->struct_size != (int)sizeof(jsweep_options)) {
        set_error("jsweep_options.struct_size=%d, expected %d", opt->struct_size,
                  (int)sizeof(jsweep_options));
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (opt->sweep_mode < 0 || opt->sweep_mode > JSWEEP_MODE_PATCH || opt->priority < 0 ||
        opt->priority > JSWEEP_PRIO_PATCH_SLBD || opt->cluster_cells > 32 ||
        opt->cycle_search_max > 1024 || opt->blocks_per_sm > 32) {
        set_error("jsweep_options: value out of range");
        return JSWEEP_ERR_INVALID_ARG;
    }
    o->sweep_mode = opt->sweep_mode;
    o->priority = opt->priority;
    if (opt->cluster_cells > 0) o->cluster_cells = opt->cluster_cells;
    if (opt->blocks_per_sm > 0) o->blocks_per_sm = opt->blocks_per_sm;
    if (opt->octant_stagger > 0) o->octant_stagger = opt->octant_stagger;
    if (opt->spin_timeout_s > 0) o->spin_timeout_s = opt->spin_timeout_s;
    if (opt->cycle_search_max > 0) o->cycle_search_max = opt->cycle_search_max;
    o->debug_block_waits = opt->debug_block_waits ? 1 : 0;
    if (opt->layering < 0 || opt->layering > JSWEEP_LAYERS_LEVEL) {
        set_error("jsweep_options.layering=%d out of range", opt->layering);
        return JSWEEP_ERR_INVALID_ARG;
    }
    o->layering = opt->layering;
    if (opt->unit_order < 0 || opt->unit_order > 1) {
        set_error("jsweep_options.unit_order=%d out of range", opt->unit_order);
        return JSWEEP_ERR_INVALID_ARG;
    }
    o->unit_order = opt->unit_order;
    if (opt->patch_cells != 0 && (opt->patch_cells < 32 || opt->patch_cells > 4096)) {
        set_error("jsweep_options.patch_cells=%d out of range (32..4096)", opt->patch_cells);
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (opt->patch_cells > 0) o->patch_cells = opt->patch_cells;
    if (opt->eager_search_max < 0 || opt->eager_search_max > 1024) {
        set_error("jsweep_options.eager_search_max=%d out of range (0..1024)", opt->eager_search_max);
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (opt->eager_search_max > 0) o->eager_search_max = opt->eager_search_max;
    o->no_face_stream = opt->no_face_stream ? 1 : 0;
    o->tail_units = opt->tail_units;
    o->no_sweep_order_psi = opt->no_sweep_order_psi ? 1 : 0;
    if (opt->angles_per_warp != 0 && opt->angles_per_warp != 1 && opt->angles_per_warp != 2 &&
        opt->angles_per_warp != 4) {
        set_error("jsweep_options.angles_per_warp=%d (1, 2 or 4)", opt->angles_per_warp);
        return JSWEEP_ERR_INVALID_ARG;
    }
    o->angles_per_warp = opt->angles_per_warp > 0 ? opt->angles_per_warp : 1;
    return JSWEEP_OK;
}
}  // namespace js

extern "C" {

int jsweep_build_dags(jsweep_mesh_t mesh, jsweep_quad_t quad, const jsweep_options *opt,
                      void *stream, jsweep_dags_t *out) {
    clear_error();
    if (!mesh || !quad || !out) {
        set_error("jsweep_build_dags: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    Dags *d = new Dags();
    int rc = check_options(opt, &d->opt);
    if (rc != JSWEEP_OK) {
        delete d;
        return rc;
    }
    d->mesh = impl(mesh);
    d->mesh->refs.fetch_add(1);
    d->quad = impl(quad);
    d->quad->refs.fetch_add(1);
    d->N = d->mesh->N;
    d->M = d->quad->M;
    if ((double)d->N * (double)d->M >= 9.0e18) {
        delete d;
        set_error("jsweep_build_dags: problem too large");
        return JSWEEP_ERR_INVALID_ARG;
    }
    // First attempt: eager cycle searches capped at eager_search_max cells (most
    // components are a few cells; larger eager searches mostly run into cells
    // that are not peeled yet).  If that leaves a component the stalled search
    // cannot close, build again with the full cap everywhere.
    const int64_t l0 = g_kernel_launches.load();
    d->eager_cap = std::min(d->opt.eager_search_max > 0 ? d->opt.eager_search_max : 64, d->opt.cycle_search_max);
    rc = build_dags(d, (cudaStream_t)stream);
    if (rc == JSWEEP_ERR_CYCLE && d->eager_cap < d->opt.cycle_search_max) {
        Dags *d2 = new Dags();
        d2->opt = d->opt;
        d2->mesh = d->mesh;
        d2->mesh->refs.fetch_add(1);
        d2->quad = d->quad;
        d2->quad->refs.fetch_add(1);
        d2->N = d->N;
        d2->M = d->M;
        d2->eager_cap = d->opt.cycle_search_max;
        delete d;
        d = d2;
        clear_error();
        rc = build_dags(d, (cudaStream_t)stream);
    }
    d->timing.build_launches = g_kernel_launches.load() - l0;
    if (rc != JSWEEP_OK) {
        delete d;
        return rc;
    }
    *out = reinterpret_cast<jsweep_dags_t>(d);
    return JSWEEP_OK;
}

int jsweep_dags_destroy(jsweep_dags_t dags) {
    dags_release(impl(dags));  // a batch that still uses the handle keeps it alive
    return JSWEEP_OK;
}

int jsweep_dags_info(jsweep_dags_t dags, int64_t *n_dirs, int64_t *max_levels, int64_t *n_lag_total) {
    if (!dags) {
        set_error("jsweep_dags_info: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    if (n_dirs) *n_dirs = d->M;
    if (max_levels) *max_levels = d->Lmax;
    if (n_lag_total) *n_lag_total = d->T;
    return JSWEEP_OK;
}

static int check_dir(Dags *d, int64_t m) {
    if (m < 0 || m >= d->M) {
        set_error("direction %lld out of range [0, %lld)", (long long)m, (long long)d->M);
        return JSWEEP_ERR_INVALID_ARG;
    }
    return JSWEEP_OK;
}

int jsweep_dags_nlevels(jsweep_dags_t dags, int64_t m, int64_t *nlevels) {
    if (!dags || !nlevels) {
        set_error("jsweep_dags_nlevels: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    JS_TRY(check_dir(d, m));
    *nlevels = d->nlevels[m];
    return JSWEEP_OK;
}

int jsweep_dags_levels(jsweep_dags_t dags, int64_t m, int32_t *level_of_cell) {
    if (!dags || !level_of_cell) {
        set_error("jsweep_dags_levels: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    JS_TRY(check_dir(d, m));
    JS_CUDA(cudaDeviceSynchronize());
    JS_CUDA(cudaMemcpy(level_of_cell, d->level.as<int32_t>() + m * d->N, d->N * 4,
                       cudaMemcpyDeviceToHost));
    return JSWEEP_OK;
}

int jsweep_dags_order(jsweep_dags_t dags, int64_t m, int32_t *order, int32_t *level_ptr) {
    if (!dags || !order || !level_ptr) {
        set_error("jsweep_dags_order: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    JS_TRY(check_dir(d, m));
    JS_CUDA(cudaDeviceSynchronize());
    JS_CUDA(cudaMemcpy(order, d->order.as<int32_t>() + m * d->N, d->N * 4, cudaMemcpyDeviceToHost));
    JS_CUDA(cudaMemcpy(level_ptr, d->lp.as<int32_t>() + d->lp_off[m], (d->nlevels[m] + 1) * 4,
                       cudaMemcpyDeviceToHost));
    return JSWEEP_OK;
}

int jsweep_dags_schedule(jsweep_dags_t dags, int64_t m, int64_t *n_layers, int32_t *order, int32_t *layer_ptr) {
    if (!dags || !n_layers) {
        set_error("jsweep_dags_schedule: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    JS_TRY(check_dir(d, m));
    *n_layers = d->slayers[m];
    if (!order && !layer_ptr) return JSWEEP_OK;
    JS_CUDA(cudaDeviceSynchronize());
    if (order) JS_CUDA(cudaMemcpy(order, d->s_order + m * d->N, d->N * 4, cudaMemcpyDeviceToHost));
    if (layer_ptr)
        JS_CUDA(cudaMemcpy(layer_ptr, d->s_lp + d->sp_off[m], (d->slayers[m] + 1) * 4, cudaMemcpyDeviceToHost));
    return JSWEEP_OK;
}

int jsweep_dags_lagged(jsweep_dags_t dags, int64_t m, int64_t *rows, int64_t *n) {
    if (!dags || !n) {
        set_error("jsweep_dags_lagged: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    JS_TRY(check_dir(d, m));
    int64_t a = d->lag_ptr_h[m], b = d->lag_ptr_h[m + 1];
    *n = b - a;
    if (!rows || b == a) return JSWEEP_OK;
    std::vector<int32_t> f(b - a), u(b - a), v(b - a);
    JS_CUDA(cudaDeviceSynchronize());
    JS_CUDA(cudaMemcpy(f.data(), d->lag_face.as<int32_t>() + a, (b - a) * 4, cudaMemcpyDeviceToHost));
    JS_CUDA(cudaMemcpy(u.data(), d->lag_up.as<int32_t>() + a, (b - a) * 4, cudaMemcpyDeviceToHost));
    JS_CUDA(cudaMemcpy(v.data(), d->lag_dn.as<int32_t>() + a, (b - a) * 4, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < b - a; ++i) {
        rows[3 * i] = f[i];
        rows[3 * i + 1] = u[i];
        rows[3 * i + 2] = v[i];
    }
    return JSWEEP_OK;
}

int jsweep_dags_reset_lag(jsweep_dags_t dags) {
    if (!dags) {
        set_error("jsweep_dags_reset_lag: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    if (d->psi_lag.p) JS_CUDA(cudaMemset(d->psi_lag.p, 0, d->psi_lag.bytes));
    return JSWEEP_OK;
}

int jsweep_dags_set_options(jsweep_dags_t dags, const jsweep_options *opt) {
    if (!dags) {
        set_error("jsweep_dags_set_options: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    Dags *d = impl(dags);
    jsweep_options o;
    JS_TRY(check_options(opt, &o));
    d->opt = o;
    return JSWEEP_OK;
}

int jsweep_dags_timing(jsweep_dags_t dags, jsweep_timing *t) {
    if (!dags || !t) {
        set_error("jsweep_dags_timing: NULL");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *t = impl(dags)->timing;
    return JSWEEP_OK;
}

static int check_prec(int nrhs, int precision) {
    if (nrhs < 1 || nrhs > 8) {
        set_error("nrhs=%d outside 1..8", nrhs);
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (precision != JSWEEP_F64 && precision != JSWEEP_F32) {
        set_error("precision=%d is neither JSWEEP_F64 nor JSWEEP_F32", precision);
        return JSWEEP_ERR_INVALID_ARG;
    }
    return JSWEEP_OK;
}

int jsweep_sweep(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                 const void *ang_source, const void *inflow, void *phi_out, void *psi_out,
                 void *stream) {
    clear_error();
    if (!dags || !sigma_t || !ang_source || !phi_out) {
        set_error("jsweep_sweep: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_TRY(check_prec(nrhs, precision));
    const int64_t l0 = g_kernel_launches.load();
    int rc = run_sweep(impl(dags), nrhs, precision, sigma_t, ang_source, inflow, phi_out, psi_out,
                       (cudaStream_t)stream);
    impl(dags)->timing.call_launches = g_kernel_launches.load() - l0;
    return rc;
}

int jsweep_source_iterate(jsweep_dags_t dags, int nrhs, int precision, const void *sigma_t,
                          const void *c_ratio, const void *q, const void *inflow, double tol,
                          int max_iters, void *phi_out, int *iters_out, double *resid_out,
                          void *stream) {
    clear_error();
    if (!dags || !sigma_t || !c_ratio || !q || !phi_out) {
        set_error("jsweep_source_iterate: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_TRY(check_prec(nrhs, precision));
    if (!(tol >= 0.0) || max_iters < 1) {
        set_error("jsweep_source_iterate: tol=%g max_iters=%d", tol, max_iters);
        return JSWEEP_ERR_INVALID_ARG;
    }
    const int64_t l0 = g_kernel_launches.load();
    int rc = run_source_iteration(impl(dags), nrhs, precision, sigma_t, c_ratio, q, inflow, tol,
                                  max_iters, phi_out, iters_out, resid_out, (cudaStream_t)stream);
    impl(dags)->timing.call_launches = g_kernel_launches.load() - l0;
    return rc;
}

int jsweep_bounds_checked(void) {
#ifdef JSWEEP_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

int jsweep_bounds_error(uint64_t *word) {
    clear_error();
    if (!word) {
        set_error("jsweep_bounds_error: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    *word = 0;
    unsigned long long *w = bounds_word();
    if (!w) return JSWEEP_OK;
    unsigned long long v = 0;
    JS_CUDA(cudaDeviceSynchronize());
    JS_CUDA(cudaMemcpy(&v, w, 8, cudaMemcpyDeviceToHost));
    JS_CUDA(cudaMemset(w, 0, 8));
    *word = v;
    return JSWEEP_OK;
}

int jsweep_source_iterate_mg(jsweep_dags_t dags, int n_groups, int precision, const void *sigma_t,
                             const void *sigma_s, const void *q, const void *inflow, double tol, int max_iters,
                             void *phi_out, int *iters_out, double *resid_out, void *stream) {
    clear_error();
    if (!dags || !sigma_t || !sigma_s || !q || !phi_out) {
        set_error("jsweep_source_iterate_mg: NULL argument");
        return JSWEEP_ERR_INVALID_ARG;
    }
    if (n_groups < 1 || n_groups > 8) {
        set_error("jsweep_source_iterate_mg: n_groups=%d outside 1..8", n_groups);
        return JSWEEP_ERR_INVALID_ARG;
    }
    JS_TRY(check_prec(1, precision));
    if (!(tol >= 0.0) || max_iters < 1) {
        set_error("jsweep_source_iterate_mg: tol=%g max_iters=%d", tol, max_iters);
        return JSWEEP_ERR_INVALID_ARG;
    }
    const int64_t l0 = g_kernel_launches.load();
    int rc = run_source_iteration_mg(impl(dags), n_groups, precision, sigma_t, sigma_s, q, inflow, tol, max_iters,
                                     phi_out, iters_out, resid_out, (cudaStream_t)stream);
    impl(dags)->timing.call_launches = g_kernel_launches.load() - l0;
    return rc;
}

}  // extern "C"
