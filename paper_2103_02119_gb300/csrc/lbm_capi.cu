// lbm_capi.cu -- the C ABI of include/lbm.h: parameter validation, device
// memory, kernel dispatch and host <-> device transfers.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "dev_alloc.h"
#include "lbm.h"
#include "lbm_launch.h"
#include "nvtx_range.h"

using lbm::AuxParams;
using lbm::CollConst;
using lbm::DiagPartial;
using lbm::KParams;

// Countdown of lbm_debug_fail_alloc: when it is n > 0, the n-th device
// allocation from then on fails.
static std::atomic<long long> g_fail_alloc{0};

cudaError_t lbm::dev_malloc(void** p, size_t bytes) {
    long long n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

static unsigned long long next_handle_serial() {
    static std::atomic<unsigned long long> n{0};
    return ++n;
}

struct lbm_handle {
    lbm_params p{};
    int pitch = 0;
    long long plane = 0;       // element stride between population planes
    int rstride = 0;           // element stride between rows of a plane
    long long N = 0;           // nx * ny
    long long n_fluid = 0;
    cudaStream_t stream = nullptr;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t* lmask = nullptr;  // device link mask (nullable)
    double* uprev = nullptr;   // 2N doubles, residual reference
    int have_prev = 0;
    int64_t prev_step = 0;
    double* stage = nullptr;   // host <-> device staging (doubles)
    size_t stage_elems = 0;
    DiagPartial* part = nullptr;
    int* status = nullptr;     // device word set by a step kernel that timed out
    bool owns_status = true;   // false for a view of a batch lattice
    unsigned wait_limit = lbm::kWaitPolls;  // polls of the step kernel's row wait
    int diag_blocks = 0;
    int bx = 0, nbands = 0;
    int64_t steps = 0, launches = 0;
    void* dfield = nullptr;    // small lattices: the density field of a step
    bool small = false;        // steps run as one cluster launch (small_step.cu)
    cudaStream_t cap = nullptr;                     // owned, for graph capture only
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // runs of steps from f[0] / f[1]
    char err[512] = {0};
    unsigned long long serial = next_handle_serial();
};

namespace {

thread_local char g_err[512] = "no error";

// Population layout of every handle (see lbm_device.cuh).
constexpr bool kRowInterleaved = false;
// steps per launch of the small-lattice kernel (bounds one launch to a few ms)
constexpr int kSmallRun = 1024;

void set_err(lbm_handle* h, const char* fmt, ...) {
    char* dst = h ? h->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

lbm_status cuda_fail(lbm_handle* h, cudaError_t e, const char* what) {
    set_err(h, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(h, call, what)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

size_t elem_size(const lbm_handle* h) { return h->p.precision == 64 ? 8 : 4; }
size_t buf_bytes(const lbm_handle* h) {
    return 9 * (size_t)h->pitch * (size_t)h->p.ny * elem_size(h);
}

bool is_fin(double v) { return std::isfinite(v); }

// Rest equilibrium weights of the rectangular D2Q9 lattice: the product of
// the 1-D factors (1 - cs2, cs2/2, cs2/2) along x and
// (1 - cs2/a^2, cs2/(2a^2), cs2/(2a^2)) along y.
void rest_weights(double a, double cs2, double w[9]) {
    const double wx[3] = {1.0 - cs2, 0.5 * cs2, 0.5 * cs2};
    const double wy[3] = {1.0 - cs2 / (a * a), 0.5 * cs2 / (a * a), 0.5 * cs2 / (a * a)};
    for (int i = 0; i < 9; ++i) {
        const int sx = lbm::ex(i), sy = lbm::ey(i);
        w[i] = wx[sx == 0 ? 0 : (sx > 0 ? 1 : 2)] * wy[sy == 0 ? 0 : (sy > 0 ? 1 : 2)];
    }
}

const char* validate(const lbm_params* p) {
    if (!p) return "params is NULL";
    if (p->nx < 3 || p->ny < 3) return "nx and ny must be >= 3";
    if ((double)p->nx * (double)p->ny > 4.0e9) return "nx*ny too large";
    if (!is_fin(p->a) || !(p->a > 0.0)) return "a must be finite and > 0";
    if (!is_fin(p->cs2) || !(p->cs2 > 0.0) || !(p->cs2 < 1.0) || !(p->cs2 < p->a * p->a))
        return "cs2 must satisfy 0 < cs2 < min(1, a^2)";
    for (int j = 0; j < 9; ++j)
        if (!is_fin(p->omega[j]) || p->omega[j] < 0.0 || p->omega[j] > 2.0)
            return "every omega must lie in [0, 2]";
    if (!(p->omega[3] > 0.0) || !(p->omega[4] > 0.0)) return "omega[3] and omega[4] must be > 0";
    if (!is_fin(p->Fx) || !is_fin(p->Fy)) return "force must be finite";
    if (!is_fin(p->rho0) || p->rho0 < 0.0) return "rho0 must be finite and >= 0";
    if (p->precision != 32 && p->precision != 64) return "precision must be 32 or 64";
    if ((p->periodic_x != 0 && p->periodic_x != 1) || (p->periodic_y != 0 && p->periodic_y != 1))
        return "periodic flags must be 0 or 1";
    for (int k = 0; k < 4; ++k)
        if (!is_fin(p->wall_u[k][0]) || !is_fin(p->wall_u[k][1])) return "wall velocities must be finite";
    if ((p->use_iso_corr != 0 && p->use_iso_corr != 1) || (p->use_gi_corr != 0 && p->use_gi_corr != 1))
        return "correction flags must be 0 or 1";
    if (p->block_x != 0 && p->block_x != 32 && p->block_x != 64 && p->block_x != 128 &&
        p->block_x != 256)
        return "block_x must be 0, 32, 64, 128 or 256";
    if (p->bands < 0) return "bands must be >= 0";
    if (p->scheme != 0 && p->scheme != 1 && p->scheme != -1)
        return "scheme must be 0 (RC-LBM), 1 (RNR-LBM) or -1 (no collision)";
    // the 2x2 strain-rate system of Eq. 37-38 must be solvable at rest
    const double cs2 = p->cs2, a2 = p->a * p->a;
    const double b1 = -2 * cs2 / p->omega[3] - (1 - 3 * cs2) / 2;
    const double b2 = -2 * cs2 / p->omega[3] - (a2 - 3 * cs2) / 2;
    const double c1 = -2 * cs2 / p->omega[4] - (1 - 3 * cs2) / 2;
    const double c2 = 2 * cs2 / p->omega[4] + (a2 - 3 * cs2) / 2;
    if (!(std::fabs(b1 * c2 - b2 * c1) > 1e-12)) return "strain-rate system (Eq. 37-38) is singular";
    return nullptr;
}

// A constant as a lane value of the collision (FP32: both halves of a float2).
template <typename T>
typename lbm::Lane<T>::V lane_of(double v);
template <>
float2 lane_of<float>(double v) { return make_float2((float)v, (float)v); }
template <>
double lane_of<double>(double v) { return v; }

// Storage geometry of one lattice.
struct Geometry {
    int pitch;
    long long plane;
    int rstride;
    const uint8_t* lmask;
    int* status;
    unsigned wait_limit = lbm::kWaitPolls;
};

template <typename T>
KParams<T> kparams_of(const lbm_params& q, const Geometry& g) {
    KParams<T> k{};
    k.nx = q.nx;
    k.ny = q.ny;
    k.pitch = g.pitch;
    k.plane = g.plane;
    k.rstride = g.rstride;
    k.px = q.periodic_x;
    k.py = q.periodic_y;
    k.moving = 0;
    for (int w = 0; w < 4; ++w) {
        const bool exists = w < 2 ? !q.periodic_x : !q.periodic_y;
        if (exists && (q.wall_u[w][0] != 0.0 || q.wall_u[w][1] != 0.0)) k.moving = 1;
        k.wall_u[w][0] = T(q.wall_u[w][0]);
        k.wall_u[w][1] = T(q.wall_u[w][1]);
    }
    const double a = q.a, cs2 = q.cs2, a2 = a * a;
    k.a = T(a);
    k.iah = T(0.5 / a);
    k.iah2 = T(0.5 / a2);
    k.cs2 = T(cs2);
    k.rho0 = T(q.rho0);
    const double* w = q.omega;
    const double g1 = 1.0 - 3.0 * cs2, g2 = a2 - 3.0 * cs2;
    CollConst<T>& c = k.cc;
    auto L = [](double v) { return lane_of<T>(v); };
    c.rho0 = L(q.rho0);
    c.nrho0 = L(-q.rho0);
    c.a = L(a);
    c.a2 = L(a2);
    c.cs2 = L(cs2);
    c.cs4 = L(cs2 * cs2);
    c.Fx = L(q.Fx);
    c.Fy = L(q.Fy);
    c.hFx = L(0.5 * q.Fx);
    c.hFy = L(0.5 * q.Fy);
    c.twoFx = L(2.0 * q.Fx);
    c.twoFy = L(2.0 * q.Fy);
    c.half = L(0.5);
    c.two = L(2.0);
    c.c15 = L(1.5);
    c.nc15 = L(-1.5);
    c.b1c = L(-2.0 * cs2 / w[3] - 0.5 * g1);
    c.b2c = L(-2.0 * cs2 / w[3] - 0.5 * g2);
    c.c1c = L(-2.0 * cs2 / w[4] - 0.5 * g1);
    c.c2c = L(2.0 * cs2 / w[4] + 0.5 * g2);
    c.g1h = L(0.5 * g1);
    c.g2h = L(0.5 * g2);
    c.g1i = L(q.use_iso_corr ? g1 : 0.0);
    c.g2i = L(q.use_iso_corr ? g2 : 0.0);
    c.ng3 = L(q.use_gi_corr ? -3.0 : 0.0);
    c.lw3 = L(1.0 - 0.5 * w[3]);
    c.lw4 = L(1.0 - 0.5 * w[4]);
    c.lw5 = L(1.0 - 0.5 * w[5]);
    c.lw6 = L(1.0 - 0.5 * w[6]);
    c.lw7 = L(1.0 - 0.5 * w[7]);
    c.lw8 = L(1.0 - 0.5 * w[8]);
    c.nw3 = L(-w[3]);
    c.nw4 = L(-w[4]);
    c.nw5 = L(-w[5]);
    c.nw6 = L(-w[6]);
    c.nw7 = L(-w[7]);
    c.nw8 = L(-w[8]);
    c.iah = L(0.5 / a);
    c.niah = L(-0.5 / a);
    c.iah2 = L(0.5 / a2);
    c.nia2 = L(-1.0 / a2);
    c.qa = L(0.25 / a);
    c.nqa = L(-0.25 / a);
    c.qa2 = L(0.25 / a2);
    c.lw3h = L(0.5 - 0.25 * w[3]);
    c.lw4h = L(0.5 - 0.25 * w[4]);
    c.nw3h = L(-0.5 * w[3]);
    c.nw4h = L(-0.5 * w[4]);
    k.forced = q.Fx != 0.0 || q.Fy != 0.0;
    k.lmask = g.lmask;
    k.collide = q.scheme >= 0;
    k.raw = q.scheme == 1;
    k.status = g.status;
    k.spin_limit = g.wait_limit;
    return k;
}

AuxParams aux_of(const lbm_params& q, const Geometry& g) {
    AuxParams a{};
    a.nx = q.nx;
    a.ny = q.ny;
    a.pitch = g.pitch;
    a.plane = g.plane;
    a.rstride = g.rstride;
    a.px = q.periodic_x;
    a.py = q.periodic_y;
    a.a = q.a;
    a.cs2 = q.cs2;
    a.rho0 = q.rho0;
    a.Fx = q.Fx;
    a.Fy = q.Fy;
    double w[9];
    rest_weights(q.a, q.cs2, w);
    for (int i = 0; i < 9; ++i) a.wrest[i] = w[i] * q.rho0;
    a.w3 = q.omega[3];
    a.w4 = q.omega[4];
    a.w5 = q.omega[5];
    a.lmask = g.lmask;
    return a;
}

Geometry geometry(const lbm_handle* h) {
    return Geometry{h->pitch, h->plane, h->rstride, h->lmask, h->status, h->wait_limit};
}
template <typename T>
KParams<T> kparams(const lbm_handle* h) { return kparams_of<T>(h->p, geometry(h)); }
AuxParams aux(const lbm_handle* h) { return aux_of(h->p, geometry(h)); }

// Link mask of every cell (see lbm_device.cuh: bit i-1 = source of
// direction i is a wall or solid node, 0xFF = solid cell).  Fluid cells
// with no fluid neighbour become solid.  Returns the number of fluid cells.
long long build_link_mask(const lbm_params& p, const uint8_t* solid, int pitch,
                          std::vector<uint8_t>& out) {
    const int nx = p.nx, ny = p.ny;
    out.assign((size_t)pitch * ny, 0xFF);
    auto is_solid = [&](int x, int y) -> bool {
        if (x < 0 || x >= nx) {
            if (!p.periodic_x) return true;
            x = (x + nx) % nx;
        }
        if (y < 0 || y >= ny) {
            if (!p.periodic_y) return true;
            y = (y + ny) % ny;
        }
        return solid[(size_t)y * nx + x] != 0;
    };
    long long nf = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (solid[(size_t)y * nx + x]) continue;
            unsigned b = 0;
            for (int i = 1; i < 9; ++i)
                if (is_solid(x - lbm::ex(i), y - lbm::ey(i))) b |= 1u << (i - 1);
            out[(size_t)y * pitch + x] = (uint8_t)b;  // b == 0xFF: isolated -> solid
            if (b != 0xFFu) ++nf;
        }
    return nf;
}

lbm_status ensure_stage(lbm_handle* h, size_t elems) {
    if (h->stage_elems >= elems) return LBM_OK;
    if (h->stage) cudaFree(h->stage);
    h->stage = nullptr;
    h->stage_elems = 0;
    CK(h, lbm::dev_alloc(&h->stage, elems * sizeof(double)), "cudaMalloc(staging)");
    h->stage_elems = elems;
    return LBM_OK;
}

// Device pointers for up to `n` caller arrays of N doubles each: on_device
// arrays pass through; host arrays are uploaded into the staging buffer.
lbm_status device_inputs(lbm_handle* h, const double* const* in, int n, int on_device,
                         const double** out, size_t per) {
    if (on_device) {
        for (int i = 0; i < n; ++i) out[i] = in[i];
        return LBM_OK;
    }
    bool any = false;
    for (int i = 0; i < n; ++i) any |= in[i] != nullptr;
    if (any) {
        lbm_status s = ensure_stage(h, per * n);
        if (s != LBM_OK) return s;
    }
    for (int i = 0; i < n; ++i) {
        out[i] = nullptr;
        if (!in[i]) continue;
        CK(h, cudaMemcpyAsync(h->stage + per * i, in[i], per * sizeof(double),
                              cudaMemcpyHostToDevice, h->stream),
           "cudaMemcpyAsync(H2D)");
        out[i] = h->stage + per * i;
    }
    return LBM_OK;
}

// Steps per captured graph of a single lattice (even, so a run starts and
// ends on the same buffer).
constexpr int kRunSteps = 50;

void drop_run_graphs(lbm_handle* h) {
    for (auto& g : h->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Launches n steps from buffer `from` on stream s.
template <typename T>
cudaError_t launch_steps_of(lbm_handle* h, const KParams<T>& k, int from, int n, cudaStream_t s) {
    for (int i = 0; i < n; ++i) {
        const int c = (from + i) & 1;
        cudaError_t e = lbm::launch_step<T>((const T*)h->f[c], (T*)h->f[c ^ 1], k, h->bx,
                                            h->nbands, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The graph of kRunSteps steps starting from buffer `from`, captured once
// on the handle's own stream (the parameters are fixed in it; changing them
// drops the graphs).
template <typename T>
lbm_status ensure_run_graph(lbm_handle* h, const KParams<T>& k, int from) {
    if (h->graph[from]) return LBM_OK;
    if (!h->cap) CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    cudaError_t e = launch_steps_of<T>(h, k, from, kRunSteps, h->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e != cudaSuccess ? e : e2, "graph capture of the step");
    }
    e = cudaGraphInstantiate(&h->graph[from], g, 0);
    cudaGraphDestroy(g);
    CK(h, e, "cudaGraphInstantiate");
    return LBM_OK;
}

template <typename T>
lbm_status step_lattice(lbm_handle* h, int64_t nsteps) {
    const KParams<T> k = kparams<T>(h);
    if (h->small) {  // one cluster launch runs up to kSmallRun steps
        for (int64_t left = nsteps; left > 0;) {
            const int n = left < kSmallRun ? (int)left : kSmallRun;
            CK(h, lbm::launch_small_run<T>((T*)h->f[0], (T*)h->f[1], (T*)h->dfield, k, h->cur, n,
                                           h->stream),
               "small-lattice step kernel");
            h->cur ^= n & 1;
            h->launches += 1;
            h->steps += n;
            left -= n;
        }
        return LBM_OK;
    }
    int64_t left = nsteps;
    while (left >= kRunSteps) {
        if (lbm_status st = ensure_run_graph<T>(h, k, h->cur); st != LBM_OK) return st;
        CK(h, cudaGraphLaunch(h->graph[h->cur], h->stream), "cudaGraphLaunch");
        left -= kRunSteps;
        h->launches += kRunSteps;
        h->steps += kRunSteps;
    }
    CK(h, launch_steps_of<T>(h, k, h->cur, (int)left, h->stream), "step kernel");
    h->cur ^= (int)(left & 1);
    h->launches += left;
    h->steps += left;
    return LBM_OK;
}

// A new state: the step counter, the residual reference and the timeout
// report start again (a batch's view leaves the batch's report alone).
// The error a nonzero status word of the step kernels reports.
lbm_status status_error(lbm_handle* h, int kstatus) {
    if (kstatus & lbm::kStatusBounds) {
        set_err(h, "a device bounds check failed in a step kernel (status %d)", kstatus);
        return LBM_ERR_BOUNDS;
    }
    set_err(h, "a step kernel gave up waiting for its staged data (status %d)", kstatus);
    return LBM_ERR_TIMEOUT;
}

lbm_status reset_counters(lbm_handle* h) {
    h->steps = 0;
    h->have_prev = 0;
    h->prev_step = 0;
    if (h->owns_status && h->status)
        CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "cudaMemsetAsync(status)");
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_build_flags(void) { return lbm::kChecked ? LBM_BUILD_CHECKED : 0; }

lbm_status lbm_params_init(lbm_params* p) {
    if (!p) return LBM_ERR_INVALID;
    std::memset(p, 0, sizeof(*p));
    p->nx = 64;
    p->ny = 64;
    p->a = 1.0;
    p->cs2 = 1.0 / 3.0;
    for (int j = 0; j < 9; ++j) p->omega[j] = 1.0;
    p->rho0 = 1.0;
    p->precision = 32;
    p->periodic_x = 1;
    p->periodic_y = 1;
    p->use_iso_corr = 1;
    p->use_gi_corr = 1;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_params* p, const uint8_t* solid_mask, void* cuda_stream,
                      lbm_handle** out) {
    LBM_RANGE("lbm_create");
    if (!out) {
        set_err(nullptr, "out is NULL");
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    if (const char* why = validate(p)) {
        set_err(nullptr, "invalid parameters: %s", why);
        return LBM_ERR_INVALID;
    }
    lbm_handle* h = new (std::nothrow) lbm_handle();
    if (!h) {
        set_err(nullptr, "host allocation failed");
        return LBM_ERR_OOM;
    }
    h->p = *p;
    h->stream = (cudaStream_t)cuda_stream;
    h->pitch = (p->nx + 31) / 32 * 32;
    // plane-major layout [9][ny][pitch]; kRowInterleaved stores [ny][9][pitch]
    if (kRowInterleaved) {
        h->plane = h->pitch;
        h->rstride = 9 * h->pitch;
    } else {
        h->plane = (long long)h->pitch * p->ny;
        h->rstride = h->pitch;
    }
    h->N = (long long)p->nx * p->ny;
    h->n_fluid = h->N;

    auto fail = [&](lbm_status s) {
        std::snprintf(g_err, sizeof(g_err), "%s", h->err);
        lbm_destroy(h);
        return s;
    };
#define CKC(call, what)                                        \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return fail(cuda_fail(h, e_, what)); \
    } while (0)

    if (solid_mask) {
        std::vector<uint8_t> lm;
        h->n_fluid = build_link_mask(*p, solid_mask, h->pitch, lm);
        CKC(lbm::dev_alloc(&h->lmask, lm.size()), "cudaMalloc(link mask)");
        CKC(cudaMemcpy(h->lmask, lm.data(), lm.size(), cudaMemcpyHostToDevice),
            "cudaMemcpy(link mask)");
    }
    for (int b = 0; b < 2; ++b) {
        CKC(lbm::dev_alloc(&h->f[b], buf_bytes(h)), "cudaMalloc(distributions)");
        CKC(cudaMemsetAsync(h->f[b], 0, buf_bytes(h), h->stream), "cudaMemset");
    }
    int dev = 0, sms = 1;
    CKC(cudaGetDevice(&dev), "cudaGetDevice");
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    h->diag_blocks = 2 * sms;
    CKC(lbm::dev_alloc(&h->part, sizeof(DiagPartial) * (h->diag_blocks + 1)), "cudaMalloc(diagnostics)");
    CKC(lbm::dev_alloc(&h->status, sizeof(int)), "cudaMalloc(status)");
    CKC(cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "cudaMemset");

    // Step kernel launch shape: one block per BX columns and per band of
    // rows, sized so that every block is resident at once (one wave).
    const bool f64 = p->precision == 64;
    auto seg_width = [&](int b) {
        return f64 ? lbm::step_segment_width<double>(b) : lbm::step_segment_width<float>(b);
    };
    int bx = p->block_x;
    if (bx == 0) bx = p->nx <= seg_width(32) ? 32 : p->nx <= seg_width(64) ? 64 : 128;
    h->bx = bx;
    const int nseg = (p->nx + seg_width(bx) - 1) / seg_width(bx);
    int nb = p->bands;
    if (nb == 0) {
        // Short bands (about 14 rows) keep the blocks that run at the same
        // time on nearby rows; enough of them to fill every SM, but bands of
        // at least 6 rows so that the two extra rows a band reads stay cheap
        // -- unless even that leaves SMs idle (small lattices, whose step
        // time is one block's row march): then bands down to one row.
        const int occ = p->precision == 64 ? lbm::step_occupancy<double>(bx, solid_mask != nullptr)
                                           : lbm::step_occupancy<float>(bx, solid_mask != nullptr);
        const int fill = (occ * sms + nseg - 1) / nseg;
        const int cap = (long long)nseg * (p->ny / 6) >= sms ? p->ny / 6 : p->ny;
        nb = p->ny / 14;
        if (nb < fill) nb = fill < cap ? fill : cap;
        if (nb < 1) nb = 1;
    }
    if (nb > p->ny) nb = p->ny;
    if (nb > 65535) nb = 65535;  // grid.y limit
    h->nbands = nb;
    // small lattices: all the steps of an lbm_step call in one launch of one
    // thread-block cluster, when the device can hold it
    if (h->N <= lbm::kSmallCells && !kRowInterleaved) {
        const bool fits = f64 ? lbm::small_run_fits<double>(kparams<double>(h))
                              : lbm::small_run_fits<float>(kparams<float>(h));
        if (fits) {
            CKC(lbm::dev_alloc(&h->dfield, (size_t)h->N * elem_size(h)), "cudaMalloc(density field)");
            h->small = true;
        }
    }
#undef CKC
    lbm_status s = lbm_init_fields(h, nullptr, nullptr, nullptr, 0);
    if (s != LBM_OK) return fail(s);
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    drop_run_graphs(h);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->f[0]) cudaFree(h->f[0]);
    if (h->f[1]) cudaFree(h->f[1]);
    if (h->lmask) cudaFree(h->lmask);
    if (h->dfield) cudaFree(h->dfield);
    if (h->uprev) cudaFree(h->uprev);
    if (h->stage) cudaFree(h->stage);
    if (h->part) cudaFree(h->part);
    if (h->status) cudaFree(h->status);
    delete h;
}

lbm_status lbm_init_fields(lbm_handle* h, const double* rho, const double* ux,
                           const double* uy, int on_device) {
    LBM_RANGE("lbm_init_fields");
    if (!h) return LBM_ERR_INVALID;
    const double* in[3] = {rho, ux, uy};
    const double* d[3];
    lbm_status s = device_inputs(h, in, 3, on_device, d, (size_t)h->N);
    if (s != LBM_OK) return s;
    const AuxParams a = aux(h);
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_init<double>((double*)h->f[h->cur], a, d[0], d[1], d[2], h->stream)
                        : lbm::launch_init<float>((float*)h->f[h->cur], a, d[0], d[1], d[2], h->stream);
    CK(h, e, "init kernel");
    if (lbm_status st = reset_counters(h); st != LBM_OK) return st;
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
    LBM_RANGE("lbm_step");
    if (!h) return LBM_ERR_INVALID;
    if (nsteps < 0) {
        set_err(h, "nsteps must be >= 0");
        return LBM_ERR_INVALID;
    }
    // runs of kRunSteps steps replay a captured graph, the rest launch directly
    while (nsteps > 0) {
        const int64_t n = nsteps < (1LL << 30) ? nsteps : (1LL << 30);
        lbm_status st = h->p.precision == 64 ? step_lattice<double>(h, n) : step_lattice<float>(h, n);
        if (st != LBM_OK) return st;
        nsteps -= n;
    }
    return LBM_OK;
}

lbm_status lbm_set_small_path(lbm_handle* h, int enable) {
    if (!h) return LBM_ERR_INVALID;
    if (enable != 0 && enable != 1) {
        set_err(h, "enable must be 0 or 1");
        return LBM_ERR_INVALID;
    }
    if (enable && !h->dfield) {
        set_err(h, "this lattice has no small-lattice path (more than 4096 cells, or the cluster "
                   "does not fit the device)");
        return LBM_ERR_INVALID;
    }
    h->small = enable != 0;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_handle* h, double Fx, double Fy) {
    if (!h) return LBM_ERR_INVALID;
    if (!is_fin(Fx) || !is_fin(Fy)) {
        set_err(h, "force must be finite");
        return LBM_ERR_INVALID;
    }
    h->p.Fx = Fx;
    h->p.Fy = Fy;
    drop_run_graphs(h);  // the captured steps carry the old force
    return LBM_OK;
}

lbm_status lbm_set_wait_limit(lbm_handle* h, int64_t polls) {
    if (!h) return LBM_ERR_INVALID;
    if (polls < 0 || polls > (int64_t)lbm::kWaitPolls) {
        set_err(h, "polls must lie in [0, %u]", lbm::kWaitPolls);
        return LBM_ERR_INVALID;
    }
    h->wait_limit = (unsigned)polls;
    drop_run_graphs(h);  // the captured steps carry the old limit
    return LBM_OK;
}

lbm_status lbm_debug_fail_alloc(int64_t nth) {
    if (nth < 0) return LBM_ERR_INVALID;
    g_fail_alloc.store((long long)nth);
    return LBM_OK;
}

lbm_status lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, int on_device) {
    LBM_RANGE("lbm_moments");
    if (!h) return LBM_ERR_INVALID;
    const size_t N = (size_t)h->N;
    double* d[3] = {rho, ux, uy};
    if (!on_device) {
        lbm_status s = ensure_stage(h, 3 * N);
        if (s != LBM_OK) return s;
        for (int i = 0; i < 3; ++i) d[i] = d[i] ? h->stage + N * i : nullptr;
    }
    const AuxParams a = aux(h);
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_moments<double>((const double*)h->f[h->cur], a, d[0], d[1], d[2], h->stream)
                        : lbm::launch_moments<float>((const float*)h->f[h->cur], a, d[0], d[1], d[2], h->stream);
    CK(h, e, "moments kernel");
    if (!on_device) {
        double* outs[3] = {rho, ux, uy};
        for (int i = 0; i < 3; ++i)
            if (outs[i])
                CK(h, cudaMemcpyAsync(outs[i], d[i], N * sizeof(double), cudaMemcpyDeviceToHost,
                                      h->stream),
                   "cudaMemcpyAsync(D2H)");
        CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    }
    return LBM_OK;
}

lbm_status lbm_stress(lbm_handle* h, double* dxux, double* dyuy, double* sxy, double* txx,
                      double* tyy, double* txy, int on_device) {
    LBM_RANGE("lbm_stress");
    if (!h) return LBM_ERR_INVALID;
    const size_t N = (size_t)h->N;
    double* outs[6] = {dxux, dyuy, sxy, txx, tyy, txy};
    double* d[6];
    // staging: the density field, then (host outputs) one slot per output
    lbm_status s = ensure_stage(h, on_device ? N : 7 * N);
    if (s != LBM_OK) return s;
    double* rho = h->stage;
    for (int i = 0; i < 6; ++i)
        d[i] = (on_device || !outs[i]) ? outs[i] : h->stage + N * (i + 1);
    const AuxParams a = aux(h);
    cudaError_t e;
    if (h->p.precision == 64) {
        e = lbm::launch_moments<double>((const double*)h->f[h->cur], a, rho, nullptr, nullptr,
                                        h->stream, true);
        if (e == cudaSuccess)
            e = lbm::launch_stress<double>((const double*)h->f[h->cur], a, rho, d[0], d[1], d[2],
                                           d[3], d[4], d[5], h->stream);
    } else {
        e = lbm::launch_moments<float>((const float*)h->f[h->cur], a, rho, nullptr, nullptr,
                                       h->stream, true);
        if (e == cudaSuccess)
            e = lbm::launch_stress<float>((const float*)h->f[h->cur], a, rho, d[0], d[1], d[2],
                                          d[3], d[4], d[5], h->stream);
    }
    CK(h, e, "stress kernels");
    if (!on_device) {
        for (int i = 0; i < 6; ++i)
            if (outs[i])
                CK(h, cudaMemcpyAsync(outs[i], d[i], N * sizeof(double), cudaMemcpyDeviceToHost,
                                      h->stream),
                   "cudaMemcpyAsync(D2H)");
        CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    }
    return LBM_OK;
}

lbm_status lbm_get_f(lbm_handle* h, double* f, int on_device) {
    LBM_RANGE("lbm_get_f");
    if (!h || !f) return LBM_ERR_INVALID;
    const size_t n = 9 * (size_t)h->N;
    double* d = f;
    if (!on_device) {
        lbm_status s = ensure_stage(h, n);
        if (s != LBM_OK) return s;
        d = h->stage;
    }
    const AuxParams a = aux(h);
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_get_f<double>((const double*)h->f[h->cur], a, d, h->stream)
                        : lbm::launch_get_f<float>((const float*)h->f[h->cur], a, d, h->stream);
    CK(h, e, "get_f kernel");
    if (!on_device) {
        CK(h, cudaMemcpyAsync(f, d, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "cudaMemcpyAsync(D2H)");
        CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    }
    return LBM_OK;
}

lbm_status lbm_set_f(lbm_handle* h, const double* f, int on_device) {
    LBM_RANGE("lbm_set_f");
    if (!h || !f) return LBM_ERR_INVALID;
    const double* in[1] = {f};
    const double* d[1];
    lbm_status s = device_inputs(h, in, 1, on_device, d, 9 * (size_t)h->N);
    if (s != LBM_OK) return s;
    const AuxParams a = aux(h);
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_set_f<double>((double*)h->f[h->cur], a, d[0], h->stream)
                        : lbm::launch_set_f<float>((float*)h->f[h->cur], a, d[0], h->stream);
    CK(h, e, "set_f kernel");
    if (lbm_status st = reset_counters(h); st != LBM_OK) return st;
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return LBM_OK;
}

}  // extern "C"

namespace {

// Exact value of a fixed-point limb sum, rounded once to double.
double fixed_to_double(const long long L[lbm::kMassLimbs]) {
    constexpr int ND = lbm::kMassLimbs + 3;
    __int128 dg[ND] = {0};
    __int128 carry = 0;
    for (int k = 0; k < ND; ++k) {
        __int128 v = carry + (k < lbm::kMassLimbs ? (__int128)L[k] : 0);
        __int128 lo = v & 0xFFFFFF;
        dg[k] = lo;
        carry = (v - lo) >> 24;
    }
    // carry now holds the sign extension (0 or -1)
    bool neg = carry < 0;
    if (neg) {  // magnitude of the two's-complement digit string
        __int128 c = 1;
        for (int k = 0; k < ND; ++k) {
            __int128 v = (0xFFFFFF ^ dg[k]) + c;
            dg[k] = v & 0xFFFFFF;
            c = v >> 24;
        }
    }
    int h = ND - 1;
    while (h >= 0 && dg[h] == 0) --h;
    if (h < 0) return 0.0;
    const int lo = h - 3 < 0 ? 0 : h - 3;
    unsigned __int128 acc = 0;
    for (int k = h; k >= lo; --k) acc = (acc << 24) | (unsigned __int128)dg[k];
    bool sticky = false;
    for (int k = 0; k < lo; ++k) sticky |= dg[k] != 0;
    acc = (acc << 1) | (sticky ? 1 : 0);
    double r = std::ldexp((double)acc, 24 * lo - 1 - lbm::kMassShift);
    return neg ? -r : r;
}

}  // namespace

extern "C" {

lbm_status lbm_diagnostics(lbm_handle* h, double out[LBM_DIAG_COUNT]) {
    LBM_RANGE("lbm_diagnostics");
    if (!h || !out) return LBM_ERR_INVALID;
    if (!h->uprev) CK(h, lbm::dev_alloc(&h->uprev, 2 * (size_t)h->N * sizeof(double)), "cudaMalloc(residual)");
    const AuxParams a = aux(h);
    const int have = h->have_prev && h->steps > h->prev_step;
    // the state one step earlier is the other buffer once a step has run
    const void* prev = h->steps >= 1 ? h->f[h->cur ^ 1] : nullptr;
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_diag<double>((const double*)h->f[h->cur], (const double*)prev,
                                                   a, h->uprev, have, h->part, h->diag_blocks,
                                                   h->stream)
                        : lbm::launch_diag<float>((const float*)h->f[h->cur], (const float*)prev, a,
                                                  h->uprev, have, h->part, h->diag_blocks,
                                                  h->stream);
    CK(h, e, "diagnostics kernels");
    DiagPartial r;
    CK(h, cudaMemcpyAsync(&r, h->part + h->diag_blocks, sizeof(r), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    int kstatus = 0;
    CK(h, cudaMemcpyAsync(&kstatus, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (kstatus) return status_error(h, kstatus);
    out[0] = fixed_to_double(r.limb) + (double)h->n_fluid * h->p.rho0;
    out[1] = r.mx;
    out[2] = r.my;
    out[3] = r.en;
    out[4] = (have && r.ures > 0.0)
                 ? std::sqrt(r.dres) / ((double)(h->steps - h->prev_step) * std::sqrt(r.ures))
                 : -1.0;
    out[5] = (double)r.nonfinite;
    out[6] = (double)h->steps;
    out[7] = (prev && r.ures > 0.0) ? std::sqrt(r.sres) / std::sqrt(r.ures) : -1.0;
    h->have_prev = 1;
    h->prev_step = h->steps;
    if (r.nonfinite > 0) {
        out[0] = NAN;
        set_err(h, "%lld fluid cells hold non-finite values", (long long)r.nonfinite);
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

size_t lbm_state_bytes(const lbm_handle* h) { return h ? buf_bytes(h) : 0; }

lbm_status lbm_get_state(lbm_handle* h, void* host, size_t bytes) {
    LBM_RANGE("lbm_get_state");
    if (!h || !host) return LBM_ERR_INVALID;
    if (bytes != buf_bytes(h)) {
        set_err(h, "state buffer is %zu bytes, expected %zu", bytes, buf_bytes(h));
        return LBM_ERR_STATE;
    }
    CK(h, cudaMemcpyAsync(host, h->f[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_handle* h, const void* host, size_t bytes) {
    LBM_RANGE("lbm_set_state");
    if (!h || !host) return LBM_ERR_INVALID;
    if (bytes != buf_bytes(h)) {
        set_err(h, "state buffer is %zu bytes, expected %zu", bytes, buf_bytes(h));
        return LBM_ERR_STATE;
    }
    CK(h, cudaMemcpyAsync(h->f[h->cur], host, bytes, cudaMemcpyHostToDevice, h->stream),
       "cudaMemcpyAsync(H2D)");
    if (lbm_status st = reset_counters(h); st != LBM_OK) return st;
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return LBM_OK;
}

int64_t lbm_step_count(const lbm_handle* h) { return h ? h->steps : -1; }

int64_t lbm_launch_count(const lbm_handle* h) { return h ? h->launches : -1; }

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : g_err; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Diagnostics that allocate nothing.
//
// lbm_diagnostics allocates its residual reference field (cudaMalloc) on its
// first call.  lbm_diagnostics_noalloc computes the same values with its
// scratch -- the per-block partial sums and the reference velocity field of
// the residual -- in one fixed device array of this library instead.  The
// array is a file-scope static __device__ object: every GPU that loads the
// library holds it (kNoAllocScratchBytes, about 16.1 MiB) until the process
// exits, and every call on a device shares it.
// ---------------------------------------------------------------------------
namespace {
constexpr long long kNoAllocMaxCells = 1LL << 20;  // lattice size limit
constexpr int kNoAllocMaxBlocks = 1024;            // reduction blocks limit
constexpr size_t kNoAllocPartBytes =
    ((kNoAllocMaxBlocks + 1) * sizeof(DiagPartial) + 255) / 256 * 256;
constexpr size_t kNoAllocScratchBytes =
    kNoAllocPartBytes + 2 * (size_t)kNoAllocMaxCells * sizeof(double);
constexpr int kNoAllocMaxDevices = 128;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
// Host-side record per device: the device address of the array (its name in
// host code is only a stand-in, never a device address), and which handle's
// velocity field the reference part currently holds.
struct NoAllocDevice {
    unsigned char* base = nullptr;
    unsigned long long owner = 0;  // serial of the handle of the last call
    int64_t step = 0;              // its step counter at that call
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kNoAllocMaxDevices];
}  // namespace

extern "C" lbm_status lbm_diagnostics_noalloc(lbm_handle* h, double out[LBM_DIAG_COUNT]) {
    LBM_RANGE("lbm_diagnostics_noalloc");
    if (!h || !out) return LBM_ERR_INVALID;
    if (h->N > kNoAllocMaxCells) {
        set_err(h, "lbm_diagnostics_noalloc: the lattice has %lld cells, its fixed scratch "
                   "holds at most %lld; use lbm_diagnostics",
                (long long)h->N, (long long)kNoAllocMaxCells);
        return LBM_ERR_INVALID;
    }
    if (h->diag_blocks > kNoAllocMaxBlocks) {
        set_err(h, "lbm_diagnostics_noalloc: %d reduction blocks exceed the fixed scratch "
                   "(%d); use lbm_diagnostics",
                h->diag_blocks, kNoAllocMaxBlocks);
        return LBM_ERR_INVALID;
    }
    int dev = 0;
    CK(h, cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_err(h, "lbm_diagnostics_noalloc: device %d is beyond the %d supported", dev,
                kNoAllocMaxDevices);
        return LBM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc[dev];
    if (!d.base) {  // once per device, with that device current
        void* ptr = nullptr;
        CK(h, cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "cudaGetSymbolAddress");
        d.base = (unsigned char*)ptr;
    }
    DiagPartial* part = (DiagPartial*)d.base;
    double* uref = (double*)(d.base + kNoAllocPartBytes);
    // The reference field is valid only if this handle made the last call on
    // this device and has advanced since; nothing else needs clearing (every
    // block writes its own partial and the final sum overwrites its slot).
    const int have = d.owner == h->serial && h->steps > d.step;
    const AuxParams a = aux(h);
    const void* prev = h->steps >= 1 ? h->f[h->cur ^ 1] : nullptr;
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_diag<double>((const double*)h->f[h->cur], (const double*)prev,
                                                   a, uref, have, part, h->diag_blocks, h->stream)
                        : lbm::launch_diag<float>((const float*)h->f[h->cur], (const float*)prev, a,
                                                  uref, have, part, h->diag_blocks, h->stream);
    CK(h, e, "diagnostics kernels");
    DiagPartial r;
    CK(h, cudaMemcpyAsync(&r, part + h->diag_blocks, sizeof(r), cudaMemcpyDeviceToHost,
                          h->stream),
       "cudaMemcpyAsync(D2H)");
    int kstatus = 0;
    CK(h, cudaMemcpyAsync(&kstatus, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (kstatus) {
        // the state is not valid: no values, and no residual reference taken
        return status_error(h, kstatus);
    }
    out[0] = fixed_to_double(r.limb) + (double)h->n_fluid * h->p.rho0;
    out[1] = r.mx;
    out[2] = r.my;
    out[3] = r.en;
    out[4] = (have && r.ures > 0.0)
                 ? std::sqrt(r.dres) / ((double)(h->steps - d.step) * std::sqrt(r.ures))
                 : -1.0;
    out[5] = (double)r.nonfinite;
    out[6] = (double)h->steps;
    out[7] = (prev && r.ures > 0.0) ? std::sqrt(r.sres) / std::sqrt(r.ures) : -1.0;
    d.owner = h->serial;
    d.step = h->steps;
    if (r.nonfinite > 0) {
        out[0] = NAN;
        set_err(h, "%lld fluid cells hold non-finite values", (long long)r.nonfinite);
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Batches: many independent FP32 lattices of uneven size advanced together.
//
// Every step of a batch is one launch of the persistent batch kernel over a
// device work list of (lattice, column segment, band of rows) items of the
// active lattices; the lattice table (parameters, link mask, buffers) lives
// in device memory.  Runs of kGraphSteps steps are replayed from a CUDA
// graph captured once per (launch shape, start parity).  Residual checks
// reduce every active lattice in two launches; lattices whose residual
// reaches the tolerance are retired from the work list.
// ---------------------------------------------------------------------------
using lbm::BatchAux;
using lbm::BatchLattice;
using lbm::ResPartial;

namespace {
constexpr int kGraphSteps = 50;        // steps per captured graph (even)
constexpr int kResCellsPerBlock = 2048;  // cells per residual reduction block
}  // namespace

struct lbm_batch {
    int count = 0;
    cudaStream_t stream = nullptr;  // borrowed
    cudaStream_t cap = nullptr;     // owned, for graph capture only
    int sms = 1;
    std::vector<lbm_params> p;
    std::vector<Geometry> geo;
    std::vector<long long> N, n_fluid;
    std::vector<BatchLattice<float>> lat;  // host copy of the table
    std::vector<BatchAux> bax;
    std::vector<int> cur;                  // index into lat[k].f of the state
    std::vector<char> active, have_prev, unstable;
    std::vector<int64_t> steps, prev_step;
    std::vector<double> last_res;
    float* fbase = nullptr;
    uint8_t* mbase = nullptr;
    double* ubase = nullptr;
    BatchLattice<float>* d_lat = nullptr;
    BatchAux* d_aux = nullptr;
    // work lists, each {lattice[count], first item[count], counts[2]}: one
    // per scheme for the step (0: RC-LBM or no collision, 1: RNR-LBM), one
    // of all active lattices for the residual
    int* d_list = nullptr;
    std::vector<int> h_list;
    bool has_scheme[2] = {false, false};
    int n_active = 0, total_chunks = 0;
    bool list_dirty = true;
    int* d_two = nullptr;          // per lattice: its other buffer holds the previous step
    std::vector<int> h_two;
    ResPartial* d_part = nullptr;  // per reduction block
    ResPartial* d_res = nullptr;   // per lattice
    std::vector<ResPartial> h_res;
    DiagPartial* d_diag = nullptr; // lbm_batch_diagnostics
    int diag_blocks = 0;
    int* status = nullptr;
    double* stage = nullptr;
    size_t stage_elems = 0;
    int parity = 0;
    int bx = 32, rows = 16, grid = 0;
    // Constant-memory lattice tables (batch_table.cuh): when the active
    // lattices fit, they step in up to kBatchTables groups of one scheme
    // each, group g from table g, one group after another.
    bool table_path = true;          // use the tables when the lattices fit
    int ngroups = 0;                 // groups in use; 0: the shared-memory kernel
    int graw[lbm::kBatchTables] = {};
    int ggrid[lbm::kBatchTables] = {};
    std::vector<lbm::BatchTableLattice> gtab[lbm::kBatchTables];
    std::vector<int> gbegin[lbm::kBatchTables];  // first work item of each, then the total
    unsigned long long serial = 0;   // which batch the device's tables hold
    int device = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t launches = 0;
    char err[512] = {0};
};

namespace {

void bset_err(lbm_batch* b, const char* fmt, ...) {
    char* dst = b ? b->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
}

lbm_status bcuda_fail(lbm_batch* b, cudaError_t e, const char* what) {
    bset_err(b, "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define BCK(b, call, what)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return bcuda_fail(b, e_, what); \
    } while (0)

void drop_graphs(lbm_batch* b) {
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Work items of lattice k at the batch's launch shape.
void shape_lattice(lbm_batch* b, int k) {
    BatchLattice<float>& L = b->lat[k];
    const int W = lbm::step_segment_width<float>(b->bx);
    L.nseg = (b->p[k].nx + W - 1) / W;
    int nb = (b->p[k].ny + b->rows / 2) / b->rows;
    if (nb < 1) nb = 1;
    if (nb > b->p[k].ny) nb = b->p[k].ny;
    L.nbands = nb;
}

lbm_status set_shape(lbm_batch* b, int bx, int rows) {
    if (b->bx == bx && b->rows == rows && b->grid > 0) return LBM_OK;
    b->bx = bx;
    b->rows = rows;
    b->grid = lbm::batch_occupancy<float>(bx) * b->sms;
    for (int k = 0; k < b->count; ++k) shape_lattice(b, k);
    BCK(b, cudaMemcpyAsync(b->d_lat, b->lat.data(), sizeof(BatchLattice<float>) * b->count,
                           cudaMemcpyHostToDevice, b->stream),
        "cudaMemcpyAsync(lattice table)");
    drop_graphs(b);
    b->list_dirty = true;
    return LBM_OK;
}

// Offset of work list w (0, 1: step lists of the schemes; 2: residual list)
// in d_list / h_list.
size_t list_at(const lbm_batch* b, int w) { return (size_t)w * (2 * (size_t)b->count + 2); }

void plan_groups(lbm_batch* b);

// Uploads the work lists of the active lattices (if they changed) and plans
// the table groups.
lbm_status upload_list(lbm_batch* b) {
    if (!b->list_dirty) return LBM_OK;
    const int C = b->count;
    int n[3] = {0, 0, 0};
    long long items[3] = {0, 0, 0};
    for (int k = 0; k < C; ++k) {
        if (!b->active[k]) continue;
        const int w = b->p[k].scheme == 1 ? 1 : 0;
        int* Lw = b->h_list.data() + list_at(b, w);
        Lw[n[w]] = k;
        Lw[C + n[w]] = (int)items[w];
        items[w] += (long long)b->lat[k].nseg * b->lat[k].nbands;
        ++n[w];
        int* Lr = b->h_list.data() + list_at(b, 2);
        Lr[n[2]] = k;
        Lr[C + n[2]] = (int)items[2];
        items[2] += b->bax[k].nchunk;
        ++n[2];
    }
    for (int w = 0; w < 3; ++w) {
        if (items[w] > (1LL << 30)) {
            bset_err(b, "the batch's work list is too long");
            return LBM_ERR_INVALID;
        }
        int* Lw = b->h_list.data() + list_at(b, w);
        Lw[2 * C] = n[w];
        Lw[2 * C + 1] = (int)items[w];
    }
    BCK(b, cudaMemcpyAsync(b->d_list, b->h_list.data(), sizeof(int) * b->h_list.size(),
                           cudaMemcpyHostToDevice, b->stream),
        "cudaMemcpyAsync(work list)");
    b->n_active = n[2];
    b->total_chunks = (int)items[2];
    b->list_dirty = false;
    plan_groups(b);
    return LBM_OK;
}

// A lattice's parameters with the collision constants stored once each (the
// form of the constant-memory tables).
lbm::KParams<float, lbm::CollConstF> kparams_table(const KParams<float>& k) {
    lbm::KParams<float, lbm::CollConstF> t;
    t.nx = k.nx;
    t.ny = k.ny;
    t.pitch = k.pitch;
    t.plane = k.plane;
    t.rstride = k.rstride;
    t.px = k.px;
    t.py = k.py;
    t.moving = k.moving;
    t.collide = k.collide;
    t.raw = k.raw;
    t.forced = k.forced;
    t.spin_limit = k.spin_limit;
    t.a = k.a;
    t.iah = k.iah;
    t.iah2 = k.iah2;
    t.cs2 = k.cs2;
    t.rho0 = k.rho0;
    for (int w = 0; w < 4; ++w)
        for (int d = 0; d < 2; ++d) t.wall_u[w][d] = k.wall_u[w][d];
    t.lmask = k.lmask;
    t.status = k.status;
    t.cc = lbm::compact(k.cc);
    return t;
}

// Which batch each device's constant-memory tables hold (by batch serial;
// 0: none), and whether they hold its current groups.
std::mutex g_table_mu;
unsigned long long g_table_owner[64] = {};
bool g_table_fresh[64] = {};

// Splits the active lattices into table groups, one scheme each and at most
// kBatchTableCap lattices each, balancing their work items (largest lattice
// first to the lightest group); no groups when they do not fit in the
// tables, and the shared-memory kernel steps them instead.
void plan_groups(lbm_batch* b) {
    const int old = b->ngroups;
    int oraw[lbm::kBatchTables], ogrid[lbm::kBatchTables];
    std::copy(b->graw, b->graw + lbm::kBatchTables, oraw);
    std::copy(b->ggrid, b->ggrid + lbm::kBatchTables, ogrid);
    b->ngroups = 0;
    if (b->table_path && b->device >= 0 && b->device < 64) {
        const int cap = lbm::kBatchTableCap;
        std::vector<int> ids[2];
        for (int k = 0; k < b->count; ++k)
            if (b->active[k]) ids[b->p[k].scheme == 1 ? 1 : 0].push_back(k);
        const int need0 = ((int)ids[0].size() + cap - 1) / cap;
        const int need1 = ((int)ids[1].size() + cap - 1) / cap;
        if (need0 + need1 <= lbm::kBatchTables) {
            auto work = [&](int k) { return (long long)b->lat[k].nseg * b->lat[k].nbands; };
            int g0 = 0;
            for (int w = 0; w < 2; ++w) {
                const int ng = w == 0 ? need0 : need1;
                if (ng == 0) continue;
                std::vector<int>& v = ids[w];
                std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return work(x) > work(y); });
                std::vector<long long> load(ng, 0);
                std::vector<std::vector<int>> members(ng);
                for (int k : v) {
                    int best = -1;
                    for (int j = 0; j < ng; ++j)
                        if ((int)members[j].size() < cap && (best < 0 || load[j] < load[best]))
                            best = j;
                    members[best].push_back(k);
                    load[best] += work(k);
                }
                for (int j = 0; j < ng; ++j) {
                    // the tallest bands first: the last work items a group's
                    // blocks take are then its shortest, which shortens the
                    // kernel's tail
                    std::vector<int>& m = members[j];
                    std::stable_sort(m.begin(), m.end(), [&](int x, int y) {
                        return (long long)b->p[x].ny * b->lat[y].nbands >
                               (long long)b->p[y].ny * b->lat[x].nbands;
                    });
                    const int g = g0 + j;
                    b->gtab[g].clear();
                    b->gbegin[g].clear();
                    int at = 0;
                    for (int k : m) {
                        lbm::BatchTableLattice e;
                        e.kp = kparams_table(b->lat[k].kp);
                        e.f[0] = b->lat[k].f[0];
                        e.f[1] = b->lat[k].f[1];
                        e.nseg = b->lat[k].nseg;
                        e.nbands = b->lat[k].nbands;
                        b->gtab[g].push_back(e);
                        b->gbegin[g].push_back(at);
                        at += (int)work(k);
                    }
                    b->gbegin[g].push_back(at);
                    b->graw[g] = w;
                    b->ggrid[g] = lbm::batch_table_occupancy(g, b->bx) * b->sms;
                }
                g0 += ng;
            }
            b->ngroups = g0;
        }
    }
    // the captured graphs hold the groups' launches: a new set of groups
    // (not new table contents) needs new graphs
    bool same = old == b->ngroups;
    for (int g = 0; same && g < b->ngroups; ++g)
        same = oraw[g] == b->graw[g] && ogrid[g] == b->ggrid[g];
    if (!same) drop_graphs(b);
    std::lock_guard<std::mutex> lk(g_table_mu);
    if (b->device >= 0 && b->device < 64 && g_table_owner[b->device] == b->serial)
        g_table_fresh[b->device] = false;
}

// Makes the device's tables hold this batch's groups.  Another batch's
// kernels may still read them: the device is synchronised first then.
lbm_status ensure_tables(lbm_batch* b) {
    if (b->ngroups == 0) return LBM_OK;
    std::lock_guard<std::mutex> lk(g_table_mu);
    const int d = b->device;
    if (g_table_owner[d] == b->serial && g_table_fresh[d]) return LBM_OK;
    if (g_table_owner[d] != 0 && g_table_owner[d] != b->serial)
        BCK(b, cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    for (int g = 0; g < b->ngroups; ++g)
        BCK(b, lbm::batch_table_upload(g, b->gtab[g].data(), b->gbegin[g].data(),
                                       (int)b->gtab[g].size(), b->stream),
            "upload of a batch lattice table");
    g_table_owner[d] = b->serial;
    g_table_fresh[d] = true;
    return LBM_OK;
}

int kernels_per_step(const lbm_batch* b) {
    return b->ngroups ? b->ngroups : (int)b->has_scheme[0] + (int)b->has_scheme[1];
}

cudaError_t launch_steps(lbm_batch* b, int n, int parity, cudaStream_t s) {
    if (b->ngroups) {
        // the groups one after another on s: run side by side on streams of
        // their own they measured slower (25-31k against 38-40k MLUPS on the
        // 512-lattice sweep), each SM then holding blocks of four modules'
        // copies of the kernel
        cudaError_t e = cudaSuccess;
        for (int i = 0; e == cudaSuccess && i < n; ++i)
            for (int g = 0; e == cudaSuccess && g < b->ngroups; ++g)
                e = lbm::batch_table_launch(g, (parity + i) & 1, b->bx, b->ggrid[g], b->graw[g], s);
        return e;
    }
    const int C = b->count;
    for (int i = 0; i < n; ++i)
        for (int w = 0; w < 2; ++w) {
            if (!b->has_scheme[w]) continue;
            const int* Lw = b->d_list + list_at(b, w);
            cudaError_t e = lbm::launch_batch_step<float>(b->d_lat, Lw, Lw + C, Lw + 2 * C,
                                                          (parity + i) & 1, b->bx, b->grid, w,
                                                          s);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

lbm_status ensure_graph(lbm_batch* b, int parity) {
    if (b->graph[parity]) return LBM_OK;
    BCK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture");
    cudaError_t e = launch_steps(b, kGraphSteps, parity, b->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda_fail(b, e != cudaSuccess ? e : e2, "graph capture of the batch step");
    }
    e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    BCK(b, e, "cudaGraphInstantiate");
    return LBM_OK;
}

// A handle that views lattice k of a batch, for the single-lattice read-out
// and set-up entry points.  It owns nothing; release_view hands the staging
// buffer (which those entry points may grow) back to the batch.
void make_view(lbm_batch* b, int k, lbm_handle& h) {
    h.p = b->p[k];
    h.pitch = b->geo[k].pitch;
    h.plane = b->geo[k].plane;
    h.rstride = b->geo[k].rstride;
    h.N = b->N[k];
    h.n_fluid = b->n_fluid[k];
    h.stream = b->stream;
    h.f[0] = b->lat[k].f[b->cur[k]];
    h.f[1] = nullptr;
    h.cur = 0;
    h.lmask = const_cast<uint8_t*>(b->geo[k].lmask);
    h.stage = b->stage;
    h.stage_elems = b->stage_elems;
    h.part = b->d_diag;
    h.diag_blocks = b->diag_blocks;
    h.status = b->status;
    h.owns_status = false;
    h.steps = b->steps[k];
}

lbm_status release_view(lbm_batch* b, lbm_handle& h, lbm_status s) {
    b->stage = h.stage;
    b->stage_elems = h.stage_elems;
    if (s != LBM_OK) std::snprintf(b->err, sizeof(b->err), "%s", h.err);
    return s;
}

bool bad_index(lbm_batch* b, int k) {
    if (!b) return true;
    if (k < 0 || k >= b->count) {
        bset_err(b, "lattice index %d outside [0, %d)", k, b->count);
        return true;
    }
    return false;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_params* params, int count,
                            const uint8_t* const* solid_masks, void* cuda_stream,
                            lbm_batch** out) {
    LBM_RANGE("lbm_batch_create");
    if (!out) {
        set_err(nullptr, "out is NULL");
        return LBM_ERR_INVALID;
    }
    *out = nullptr;
    if (!params || count < 1 || count > (1 << 20)) {
        set_err(nullptr, "a batch needs 1 to 2^20 lattice parameter sets");
        return LBM_ERR_INVALID;
    }
    for (int k = 0; k < count; ++k) {
        const lbm_params& q = params[k];
        const char* why = validate(&q);
        if (!why && q.precision != 32) why = "batches hold FP32 lattices only (precision 32)";
        if (!why && 9LL * ((q.nx + 31) / 32 * 32) * q.ny >= (1LL << 31))
            why = "a lattice of a batch must hold fewer than 2^31 values per buffer";
        if (why) {
            set_err(nullptr, "invalid parameters of lattice %d: %s", k, why);
            return LBM_ERR_INVALID;
        }
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) {
        set_err(nullptr, "host allocation failed");
        return LBM_ERR_OOM;
    }
    auto fail = [&](lbm_status s) {
        std::snprintf(g_err, sizeof(g_err), "%s", b->err);
        lbm_batch_destroy(b);
        return s;
    };
#define BCKC(call, what)                                            \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return fail(bcuda_fail(b, e_, what)); \
    } while (0)
    b->count = count;
    b->stream = (cudaStream_t)cuda_stream;
    b->p.assign(params, params + count);
    b->geo.resize(count);
    b->N.resize(count);
    b->n_fluid.resize(count);
    b->lat.resize(count);
    b->bax.resize(count);
    b->cur.assign(count, 0);
    b->active.assign(count, 1);
    b->have_prev.assign(count, 0);
    b->unstable.assign(count, 0);
    b->steps.assign(count, 0);
    b->prev_step.assign(count, 0);
    b->last_res.assign(count, -1.0);
    b->h_list.assign(3 * (2 * (size_t)count + 2), 0);
    b->h_res.resize(count);

    // one allocation each for the populations (two buffers per lattice), the
    // link masks and the residual reference fields; 256-byte aligned parts
    auto up = [](size_t v, size_t a) { return (v + a - 1) / a * a; };
    std::vector<size_t> foff(count), moff(count), uoff(count);
    size_t fl = 0, ml = 0, ul = 0;
    long long chunks = 0;
    for (int k = 0; k < count; ++k) {
        const lbm_params& q = params[k];
        Geometry& g = b->geo[k];
        g.pitch = (q.nx + 31) / 32 * 32;
        g.plane = (long long)g.pitch * q.ny;
        g.rstride = g.pitch;
        b->N[k] = (long long)q.nx * q.ny;
        foff[k] = fl;
        fl += 2 * up(9 * (size_t)g.plane, 64);
        moff[k] = ml;
        ml += up((size_t)g.plane, 256);
        uoff[k] = ul;
        ul += up(2 * (size_t)b->N[k], 32);
        b->bax[k].nchunk = (int)((b->N[k] + kResCellsPerBlock - 1) / kResCellsPerBlock);
        b->bax[k].pbegin = (int)chunks;
        chunks += b->bax[k].nchunk;
    }
    if (chunks > (1LL << 30)) {
        bset_err(b, "the batch is too large");
        return fail(LBM_ERR_INVALID);
    }
    int dev = 0;
    BCKC(cudaGetDevice(&dev), "cudaGetDevice");
    BCKC(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev),
         "cudaDeviceGetAttribute");
    BCKC(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "cudaStreamCreate");
    b->device = dev;
    b->serial = next_handle_serial();

    BCKC(lbm::dev_alloc(&b->fbase, fl * sizeof(float)), "cudaMalloc(distributions)");
    BCKC(lbm::dev_alloc(&b->mbase, ml), "cudaMalloc(link masks)");
    BCKC(lbm::dev_alloc(&b->ubase, ul * sizeof(double)), "cudaMalloc(residual fields)");
    BCKC(cudaMemsetAsync(b->fbase, 0, fl * sizeof(float), b->stream), "cudaMemset");
    BCKC(cudaMemsetAsync(b->ubase, 0, ul * sizeof(double), b->stream), "cudaMemset");
    BCKC(lbm::dev_alloc(&b->status, sizeof(int)), "cudaMalloc(status)");
    BCKC(cudaMemsetAsync(b->status, 0, sizeof(int), b->stream), "cudaMemset");
    BCKC(lbm::dev_alloc(&b->d_lat, sizeof(BatchLattice<float>) * count), "cudaMalloc(lattice table)");
    BCKC(lbm::dev_alloc(&b->d_aux, sizeof(BatchAux) * count), "cudaMalloc(lattice table)");
    BCKC(lbm::dev_alloc(&b->d_list, sizeof(int) * b->h_list.size()), "cudaMalloc(work list)");
    for (int k = 0; k < count; ++k) b->has_scheme[params[k].scheme == 1 ? 1 : 0] = true;
    BCKC(lbm::dev_alloc(&b->d_part, sizeof(ResPartial) * (size_t)chunks), "cudaMalloc(residual sums)");
    BCKC(lbm::dev_alloc(&b->d_res, sizeof(ResPartial) * (size_t)count), "cudaMalloc(residual sums)");
    BCKC(lbm::dev_alloc(&b->d_two, sizeof(int) * (size_t)count), "cudaMalloc(residual flags)");
    b->h_two.assign(count, 0);
    b->diag_blocks = 2 * b->sms;
    BCKC(lbm::dev_alloc(&b->d_diag, sizeof(DiagPartial) * (b->diag_blocks + 1)),
         "cudaMalloc(diagnostics)");

    std::vector<uint8_t> zero, lm;
    for (int k = 0; k < count; ++k) {
        const lbm_params& q = params[k];
        Geometry& g = b->geo[k];
        const uint8_t* solid = solid_masks ? solid_masks[k] : nullptr;
        if (!solid) {
            zero.assign((size_t)b->N[k], 0);
            solid = zero.data();
        }
        b->n_fluid[k] = build_link_mask(q, solid, g.pitch, lm);
        uint8_t* dm = b->mbase + moff[k];
        BCKC(cudaMemcpy(dm, lm.data(), lm.size(), cudaMemcpyHostToDevice), "cudaMemcpy(link mask)");
        g.lmask = dm;
        g.status = b->status;
        BatchLattice<float>& L = b->lat[k];
        L.kp = kparams_of<float>(q, g);
        L.f[0] = b->fbase + foff[k];
        L.f[1] = b->fbase + foff[k] + up(9 * (size_t)g.plane, 64);
        b->bax[k].a = aux_of(q, g);
        b->bax[k].uprev = b->ubase + uoff[k];
    }
    BCKC(cudaMemcpyAsync(b->d_aux, b->bax.data(), sizeof(BatchAux) * count,
                         cudaMemcpyHostToDevice, b->stream),
         "cudaMemcpyAsync(lattice table)");
    b->grid = 0;
    if (lbm_status s = set_shape(b, 32, 16); s != LBM_OK) return fail(s);
    for (int k = 0; k < count; ++k)
        if (lbm_status s = lbm_batch_init_fields(b, k, nullptr, nullptr, nullptr, 1); s != LBM_OK)
            return fail(s);
    BCKC(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
#undef BCKC
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    drop_graphs(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    {
        // the device's tables no longer hold a live batch
        std::lock_guard<std::mutex> lk(g_table_mu);
        if (b->device >= 0 && b->device < 64 && g_table_owner[b->device] == b->serial) {
            g_table_owner[b->device] = 0;
            g_table_fresh[b->device] = false;
        }
    }
    cudaFree(b->fbase);
    cudaFree(b->mbase);
    cudaFree(b->ubase);
    cudaFree(b->d_lat);
    cudaFree(b->d_aux);
    cudaFree(b->d_list);
    cudaFree(b->d_part);
    cudaFree(b->d_res);
    cudaFree(b->d_two);
    cudaFree(b->d_diag);
    cudaFree(b->status);
    cudaFree(b->stage);
    delete b;
}

int lbm_batch_count(const lbm_batch* b) { return b ? b->count : -1; }

lbm_status lbm_batch_init_fields(lbm_batch* b, int k, const double* rho, const double* ux,
                                 const double* uy, int on_device) {
    LBM_RANGE("lbm_batch_init_fields");
    if (bad_index(b, k)) return LBM_ERR_INVALID;
    lbm_handle h;
    make_view(b, k, h);
    lbm_status s = release_view(b, h, lbm_init_fields(&h, rho, ux, uy, on_device));
    if (s != LBM_OK) return s;
    b->steps[k] = 0;
    b->have_prev[k] = 0;
    b->prev_step[k] = 0;
    b->unstable[k] = 0;
    b->last_res[k] = -1.0;
    return LBM_OK;
}

lbm_status lbm_batch_set_active(lbm_batch* b, int k, int on) {
    if (bad_index(b, k)) return LBM_ERR_INVALID;
    if ((b->active[k] != 0) == (on != 0)) return LBM_OK;
    if (on && b->cur[k] != b->parity) {
        // the active lattices step from f[parity]: swap this one's buffers
        BatchLattice<float>& L = b->lat[k];
        float* t = L.f[0];
        L.f[0] = L.f[1];
        L.f[1] = t;
        b->cur[k] = b->parity;
        BCK(b, cudaMemcpyAsync(b->d_lat + k, &L, sizeof(L), cudaMemcpyHostToDevice, b->stream),
            "cudaMemcpyAsync(lattice table)");
    }
    b->active[k] = on != 0;
    b->list_dirty = true;
    return LBM_OK;
}

int lbm_batch_is_active(const lbm_batch* b, int k) {
    return (b && k >= 0 && k < b->count) ? (int)b->active[k] : -1;
}

lbm_status lbm_batch_set_shape(lbm_batch* b, int block_x, int rows_per_band) {
    if (!b) return LBM_ERR_INVALID;
    if (block_x != 32 && block_x != 64 && block_x != 128) {
        bset_err(b, "block_x must be 32, 64 or 128");
        return LBM_ERR_INVALID;
    }
    if (rows_per_band < 1 || rows_per_band > 1 << 16) {
        bset_err(b, "rows_per_band must lie in [1, 65536]");
        return LBM_ERR_INVALID;
    }
    return set_shape(b, block_x, rows_per_band);
}

lbm_status lbm_batch_set_wait_limit(lbm_batch* b, int64_t polls) {
    if (!b) return LBM_ERR_INVALID;
    if (polls < 0 || polls > (int64_t)lbm::kWaitPolls) {
        bset_err(b, "polls must lie in [0, %u]", lbm::kWaitPolls);
        return LBM_ERR_INVALID;
    }
    for (int k = 0; k < b->count; ++k) {
        b->geo[k].wait_limit = (unsigned)polls;
        b->lat[k].kp.spin_limit = (unsigned)polls;
    }
    b->list_dirty = true;  // the lattice tables carry the limit too
    BCK(b, cudaMemcpyAsync(b->d_lat, b->lat.data(), sizeof(BatchLattice<float>) * b->count,
                           cudaMemcpyHostToDevice, b->stream),
        "cudaMemcpyAsync(lattice table)");
    return LBM_OK;
}

lbm_status lbm_batch_set_table_path(lbm_batch* b, int enable) {
    if (!b) return LBM_ERR_INVALID;
    if (enable != 0 && enable != 1) {
        bset_err(b, "enable must be 0 or 1");
        return LBM_ERR_INVALID;
    }
    b->table_path = enable != 0;
    b->list_dirty = true;
    return LBM_OK;
}

int lbm_batch_table_groups(lbm_batch* b) {
    if (!b) return -1;
    if (upload_list(b) != LBM_OK) return -1;
    return b->ngroups;
}

lbm_status lbm_batch_get_shape(const lbm_batch* b, int* block_x, int* rows_per_band) {
    if (!b) return LBM_ERR_INVALID;
    if (block_x) *block_x = b->bx;
    if (rows_per_band) *rows_per_band = b->rows;
    return LBM_OK;
}

}  // extern "C"

namespace {
// nsteps steps of every active lattice; runs of kGraphSteps replay a graph
// when `graphs` is set, the rest are launched one by one.
lbm_status advance(lbm_batch* b, int64_t nsteps, bool graphs) {
    if (lbm_status s = upload_list(b); s != LBM_OK) return s;
    if (b->n_active == 0 || nsteps == 0) return LBM_OK;
    if (lbm_status s = ensure_tables(b); s != LBM_OK) return s;
    int64_t left = nsteps;
    while (graphs && left >= kGraphSteps) {
        if (lbm_status s = ensure_graph(b, b->parity); s != LBM_OK) return s;
        BCK(b, cudaGraphLaunch(b->graph[b->parity], b->stream), "cudaGraphLaunch");
        left -= kGraphSteps;
        b->launches += kGraphSteps * kernels_per_step(b);
    }
    while (left > 0) {
        const int n = left < (1 << 20) ? (int)left : (1 << 20);
        BCK(b, launch_steps(b, n, (int)((b->parity + (nsteps - left)) & 1), b->stream),
            "batch step kernel");
        b->launches += n * kernels_per_step(b);
        left -= n;
    }
    b->parity = (int)((b->parity + nsteps) & 1);
    for (int k = 0; k < b->count; ++k)
        if (b->active[k]) {
            b->steps[k] += nsteps;
            b->cur[k] = b->parity;
        }
    return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
    LBM_RANGE("lbm_batch_step");
    if (!b) return LBM_ERR_INVALID;
    if (nsteps < 0) {
        bset_err(b, "nsteps must be >= 0");
        return LBM_ERR_INVALID;
    }
    return advance(b, nsteps, true);
}

lbm_status lbm_batch_residuals(lbm_batch* b, double* res) {
    LBM_RANGE("lbm_batch_residuals");
    if (!b) return LBM_ERR_INVALID;
    if (lbm_status s = upload_list(b); s != LBM_OK) return s;
    const int C = b->count;
    int kstatus = 0;
    if (b->n_active > 0) {
        // a lattice stepped since its last init holds its previous state in
        // its other buffer: its residual is then on the two-step mean
        for (int k = 0; k < C; ++k) b->h_two[k] = b->steps[k] >= 1;
        BCK(b, cudaMemcpyAsync(b->d_two, b->h_two.data(), sizeof(int) * C, cudaMemcpyHostToDevice,
                               b->stream),
            "cudaMemcpyAsync(residual flags)");
        const int* Lr = b->d_list + list_at(b, 2);
        BCK(b, lbm::launch_batch_residual(b->d_lat, b->d_aux, Lr, Lr + C, Lr + 2 * C, b->d_two,
                                          b->parity, b->d_part, b->d_res, b->n_active,
                                          b->total_chunks, b->stream),
            "batch residual kernels");
        BCK(b, cudaMemcpyAsync(b->h_res.data(), b->d_res, sizeof(ResPartial) * C,
                               cudaMemcpyDeviceToHost, b->stream),
            "cudaMemcpyAsync(D2H)");
    }
    BCK(b, cudaMemcpyAsync(&kstatus, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
        "cudaMemcpyAsync(D2H)");
    BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
    if (kstatus) {
        // reported once: the word is cleared, and the lattices that were
        // active in the steps since the last check hold invalid states
        BCK(b, cudaMemsetAsync(b->status, 0, sizeof(int), b->stream), "cudaMemsetAsync(status)");
        BCK(b, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
        if (kstatus & lbm::kStatusBounds) {
            bset_err(b, "a device bounds check failed in a batch step kernel (status %d)",
                     kstatus);
            return LBM_ERR_BOUNDS;
        }
        bset_err(b, "a batch step kernel gave up waiting for its staged data (status %d)", kstatus);
        return LBM_ERR_TIMEOUT;
    }
    int bad = 0;
    for (int k = 0; k < C; ++k) {
        if (b->active[k]) {
            const ResPartial& r = b->h_res[k];
            double R = -1.0;
            if (r.nonfinite > 0) {
                R = NAN;
                b->unstable[k] = 1;
            } else if (b->have_prev[k] && b->steps[k] > b->prev_step[k] && r.ures > 0.0) {
                R = std::sqrt(r.dres) /
                    ((double)(b->steps[k] - b->prev_step[k]) * std::sqrt(r.ures));
            }
            b->last_res[k] = R;
            b->have_prev[k] = 1;
            b->prev_step[k] = b->steps[k];
        }
        bad += b->unstable[k];
        if (res) res[k] = b->last_res[k];
    }
    if (bad) {
        bset_err(b, "%d lattices hold non-finite values", bad);
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch* b, double tol, int64_t check_every, int64_t max_steps,
                         double* res) {
    LBM_RANGE("lbm_batch_run");
    if (!b) return LBM_ERR_INVALID;
    if (!(tol >= 0.0) || check_every < 1 || max_steps < 0) {
        bset_err(b, "need tol >= 0, check_every >= 1 and max_steps >= 0");
        return LBM_ERR_INVALID;
    }
    // a first check sets the reference velocity of every active lattice
    lbm_status s = lbm_batch_residuals(b, nullptr);
    if (s != LBM_OK && s != LBM_ERR_UNSTABLE) return s;
    bool unstable = s == LBM_ERR_UNSTABLE;
    for (int k = 0; k < b->count; ++k)
        if (b->active[k] && b->unstable[k]) lbm_batch_set_active(b, k, 0);
    int64_t done = 0;
    while (done < max_steps) {
        bool any = false;
        for (int k = 0; k < b->count; ++k) any |= b->active[k] != 0;
        if (!any) break;
        const int64_t n = max_steps - done < check_every ? max_steps - done : check_every;
        if ((s = lbm_batch_step(b, n)) != LBM_OK) return s;
        done += n;
        s = lbm_batch_residuals(b, nullptr);
        if (s != LBM_OK && s != LBM_ERR_UNSTABLE) return s;
        unstable |= s == LBM_ERR_UNSTABLE;
        for (int k = 0; k < b->count; ++k) {
            if (!b->active[k]) continue;
            const double R = b->last_res[k];
            if (b->unstable[k] || (R >= 0.0 && R <= tol))
                if ((s = lbm_batch_set_active(b, k, 0)) != LBM_OK) return s;
        }
    }
    if (res)
        for (int k = 0; k < b->count; ++k) res[k] = b->last_res[k];
    if (unstable) {
        int bad = 0;
        for (int k = 0; k < b->count; ++k) bad += b->unstable[k];
        bset_err(b, "%d lattices hold non-finite values (retired)", bad);
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch* b, int trial_steps, int* block_x, int* rows_per_band) {
    LBM_RANGE("lbm_batch_tune");
    if (!b) return LBM_ERR_INVALID;
    if (trial_steps < 1) {
        bset_err(b, "trial_steps must be >= 1");
        return LBM_ERR_INVALID;
    }
    static const int kBx[] = {32, 64, 128};
    // short bands for small lattices, whose step is one band's row march
    // (64 lattices of 16-32 cells a side: 12.7 us a step with one-row
    // bands, 39 us with eight)
    static const int kRows[] = {1, 2, 4, 8, 16, 32, 64};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0), "cudaEventCreate");
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return bcuda_fail(b, ce, "cudaEventCreate");
    }
    float best = 0.0f;
    int bbx = b->bx, brows = b->rows;
    lbm_status s = LBM_OK;
    for (int bx : kBx) {
        for (int rows : kRows) {
            if ((s = set_shape(b, bx, rows)) != LBM_OK) break;
            if ((s = advance(b, 1, false)) != LBM_OK) break;  // warm-up
            if ((ce = cudaEventRecord(e0, b->stream)) != cudaSuccess) break;
            if ((s = advance(b, trial_steps, false)) != LBM_OK) break;
            if ((ce = cudaEventRecord(e1, b->stream)) != cudaSuccess) break;
            if ((ce = cudaEventSynchronize(e1)) != cudaSuccess) break;
            float ms = 0.0f;
            if ((ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
            if (best == 0.0f || ms < best) {
                best = ms;
                bbx = bx;
                brows = rows;
            }
        }
        if (s != LBM_OK || ce != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != LBM_OK) return s;
    if (ce != cudaSuccess) return bcuda_fail(b, ce, "autotuner timing");
    if ((s = set_shape(b, bbx, brows)) != LBM_OK) return s;
    if (block_x) *block_x = bbx;
    if (rows_per_band) *rows_per_band = brows;
    return LBM_OK;
}

lbm_status lbm_batch_moments(lbm_batch* b, int k, double* rho, double* ux, double* uy,
                             int on_device) {
    LBM_RANGE("lbm_batch_moments");
    if (bad_index(b, k)) return LBM_ERR_INVALID;
    lbm_handle h;
    make_view(b, k, h);
    return release_view(b, h, lbm_moments(&h, rho, ux, uy, on_device));
}

lbm_status lbm_batch_get_f(lbm_batch* b, int k, double* f, int on_device) {
    LBM_RANGE("lbm_batch_get_f");
    if (bad_index(b, k)) return LBM_ERR_INVALID;
    lbm_handle h;
    make_view(b, k, h);
    return release_view(b, h, lbm_get_f(&h, f, on_device));
}

lbm_status lbm_batch_diagnostics(lbm_batch* b, int k, double out[LBM_DIAG_COUNT]) {
    LBM_RANGE("lbm_batch_diagnostics");
    if (bad_index(b, k) || !out) return LBM_ERR_INVALID;
    lbm_handle h;
    make_view(b, k, h);
    // the residual of a batch lattice comes from lbm_batch_residuals; here the
    // staging buffer stands in for the reference velocity field
    lbm_status s = ensure_stage(&h, 2 * (size_t)h.N);
    if (s != LBM_OK) return release_view(b, h, s);
    h.uprev = h.stage;
    s = lbm_diagnostics(&h, out);
    h.uprev = nullptr;
    out[4] = b->last_res[k];
    return release_view(b, h, s);
}

int64_t lbm_batch_step_count(const lbm_batch* b, int k) {
    return (b && k >= 0 && k < b->count) ? b->steps[k] : -1;
}

int64_t lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : -1; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : g_err; }

}  // extern "C"
