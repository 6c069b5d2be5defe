// lbm_capi.cu -- the C ABI of include/lbm.h: parameter validation, device
// memory, kernel dispatch and host <-> device transfers.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "lbm.h"
#include "lbm_launch.h"

using lbm::AuxParams;
using lbm::DiagPartial;
using lbm::KParams;

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
    int diag_blocks = 0;
    int bx = 0, nbands = 0;
    int64_t steps = 0, launches = 0;
    char err[512] = {0};
    unsigned long long serial = next_handle_serial();
};

namespace {

thread_local char g_err[512] = "no error";

// Population layout of every handle (see lbm_device.cuh).
constexpr bool kRowInterleaved = false;

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
    if (p->scheme != 0 && p->scheme != -1) return "scheme must be 0 (RC-LBM) or -1 (no collision)";
    // the 2x2 strain-rate system of Eq. 37-38 must be solvable at rest
    const double cs2 = p->cs2, a2 = p->a * p->a;
    const double b1 = -2 * cs2 / p->omega[3] - (1 - 3 * cs2) / 2;
    const double b2 = -2 * cs2 / p->omega[3] - (a2 - 3 * cs2) / 2;
    const double c1 = -2 * cs2 / p->omega[4] - (1 - 3 * cs2) / 2;
    const double c2 = 2 * cs2 / p->omega[4] + (a2 - 3 * cs2) / 2;
    if (!(std::fabs(b1 * c2 - b2 * c1) > 1e-12)) return "strain-rate system (Eq. 37-38) is singular";
    return nullptr;
}

template <typename T>
KParams<T> kparams(const lbm_handle* h) {
    const lbm_params& q = h->p;
    KParams<T> k{};
    k.nx = q.nx;
    k.ny = q.ny;
    k.pitch = h->pitch;
    k.plane = h->plane;
    k.rstride = h->rstride;
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
    k.ia2 = T(1.0 / a2);
    k.iah2 = T(0.5 / a2);
    k.a2 = T(a2);
    k.cs2 = T(cs2);
    k.cs4 = T(cs2 * cs2);
    k.rho0 = T(q.rho0);
    const double* w = q.omega;
    k.w3 = T(w[3]);
    k.w4 = T(w[4]);
    k.w5 = T(w[5]);
    k.w6 = T(w[6]);
    k.w7 = T(w[7]);
    k.w8 = T(w[8]);
    k.lw3 = T(1.0 - 0.5 * w[3]);
    k.lw4 = T(1.0 - 0.5 * w[4]);
    const double g1 = 1.0 - 3.0 * cs2, g2 = a2 - 3.0 * cs2;
    k.g1i = T(q.use_iso_corr ? g1 : 0.0);
    k.g2i = T(q.use_iso_corr ? g2 : 0.0);
    k.g3 = T(q.use_gi_corr ? 3.0 : 0.0);
    k.g1h = T(0.5 * g1);
    k.g2h = T(0.5 * g2);
    k.b1c = T(-2.0 * cs2 / w[3] - 0.5 * g1);
    k.b2c = T(-2.0 * cs2 / w[3] - 0.5 * g2);
    k.c1c = T(-2.0 * cs2 / w[4] - 0.5 * g1);
    k.c2c = T(2.0 * cs2 / w[4] + 0.5 * g2);
    k.Fx = T(q.Fx);
    k.Fy = T(q.Fy);
    k.hFx = T(0.5 * q.Fx);
    k.hFy = T(0.5 * q.Fy);
    k.lmask = h->lmask;
    k.collide = q.scheme == 0;
    k.status = h->status;
    return k;
}

AuxParams aux(const lbm_handle* h) {
    AuxParams a{};
    a.nx = h->p.nx;
    a.ny = h->p.ny;
    a.pitch = h->pitch;
    a.plane = h->plane;
    a.rstride = h->rstride;
    a.px = h->p.periodic_x;
    a.py = h->p.periodic_y;
    a.a = h->p.a;
    a.cs2 = h->p.cs2;
    a.rho0 = h->p.rho0;
    a.Fx = h->p.Fx;
    a.Fy = h->p.Fy;
    double w[9];
    rest_weights(h->p.a, h->p.cs2, w);
    for (int i = 0; i < 9; ++i) a.wrest[i] = w[i] * h->p.rho0;
    a.lmask = h->lmask;
    return a;
}

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
    CK(h, cudaMalloc(&h->stage, elems * sizeof(double)), "cudaMalloc(staging)");
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

void reset_counters(lbm_handle* h) {
    h->steps = 0;
    h->have_prev = 0;
    h->prev_step = 0;
}

}  // namespace

extern "C" {

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
        CKC(cudaMalloc(&h->lmask, lm.size()), "cudaMalloc(link mask)");
        CKC(cudaMemcpy(h->lmask, lm.data(), lm.size(), cudaMemcpyHostToDevice),
            "cudaMemcpy(link mask)");
    }
    for (int b = 0; b < 2; ++b) {
        CKC(cudaMalloc(&h->f[b], buf_bytes(h)), "cudaMalloc(distributions)");
        CKC(cudaMemsetAsync(h->f[b], 0, buf_bytes(h), h->stream), "cudaMemset");
    }
    int dev = 0, sms = 1;
    CKC(cudaGetDevice(&dev), "cudaGetDevice");
    CKC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    h->diag_blocks = 2 * sms;
    CKC(cudaMalloc(&h->part, sizeof(DiagPartial) * (h->diag_blocks + 1)), "cudaMalloc(diagnostics)");
    CKC(cudaMalloc(&h->status, sizeof(int)), "cudaMalloc(status)");
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
        // at least 6 rows so that the two extra rows a band reads stay cheap.
        const int occ = p->precision == 64 ? lbm::step_occupancy<double>(bx, solid_mask != nullptr)
                                           : lbm::step_occupancy<float>(bx, solid_mask != nullptr);
        const int fill = (occ * sms + nseg - 1) / nseg;
        nb = p->ny / 14;
        if (nb < fill) nb = fill < p->ny / 6 ? fill : p->ny / 6;
        if (nb < 1) nb = 1;
    }
    if (nb > p->ny) nb = p->ny;
    if (nb > 65535) nb = 65535;  // grid.y limit
    h->nbands = nb;
#undef CKC
    lbm_status s = lbm_init_fields(h, nullptr, nullptr, nullptr, 0);
    if (s != LBM_OK) return fail(s);
    *out = h;
    return LBM_OK;
}

void lbm_destroy(lbm_handle* h) {
    if (!h) return;
    if (h->f[0]) cudaFree(h->f[0]);
    if (h->f[1]) cudaFree(h->f[1]);
    if (h->lmask) cudaFree(h->lmask);
    if (h->uprev) cudaFree(h->uprev);
    if (h->stage) cudaFree(h->stage);
    if (h->part) cudaFree(h->part);
    if (h->status) cudaFree(h->status);
    delete h;
}

lbm_status lbm_init_fields(lbm_handle* h, const double* rho, const double* ux,
                           const double* uy, int on_device) {
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
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    reset_counters(h);
    return LBM_OK;
}

lbm_status lbm_step(lbm_handle* h, int64_t nsteps) {
    if (!h) return LBM_ERR_INVALID;
    if (nsteps < 0) {
        set_err(h, "nsteps must be >= 0");
        return LBM_ERR_INVALID;
    }
    if (h->p.precision == 64) {
        const KParams<double> k = kparams<double>(h);
        for (int64_t n = 0; n < nsteps; ++n) {
            CK(h, lbm::launch_step<double>((const double*)h->f[h->cur], (double*)h->f[h->cur ^ 1],
                                           k, h->bx, h->nbands, h->stream),
               "step kernel");
            h->cur ^= 1;
            ++h->launches;
            ++h->steps;
        }
    } else {
        const KParams<float> k = kparams<float>(h);
        for (int64_t n = 0; n < nsteps; ++n) {
            CK(h, lbm::launch_step<float>((const float*)h->f[h->cur], (float*)h->f[h->cur ^ 1],
                                          k, h->bx, h->nbands, h->stream),
               "step kernel");
            h->cur ^= 1;
            ++h->launches;
            ++h->steps;
        }
    }
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
    return LBM_OK;
}

lbm_status lbm_moments(lbm_handle* h, double* rho, double* ux, double* uy, int on_device) {
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

lbm_status lbm_get_f(lbm_handle* h, double* f, int on_device) {
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
    if (!on_device) CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    reset_counters(h);
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
    if (!h || !out) return LBM_ERR_INVALID;
    if (!h->uprev) CK(h, cudaMalloc(&h->uprev, 2 * (size_t)h->N * sizeof(double)), "cudaMalloc(residual)");
    const AuxParams a = aux(h);
    const int have = h->have_prev && h->steps > h->prev_step;
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_diag<double>((const double*)h->f[h->cur], a, h->uprev, have,
                                                   h->part, h->diag_blocks, h->stream)
                        : lbm::launch_diag<float>((const float*)h->f[h->cur], a, h->uprev, have,
                                                  h->part, h->diag_blocks, h->stream);
    CK(h, e, "diagnostics kernels");
    DiagPartial r;
    CK(h, cudaMemcpyAsync(&r, h->part + h->diag_blocks, sizeof(r), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    int kstatus = 0;
    CK(h, cudaMemcpyAsync(&kstatus, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(D2H)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (kstatus) {
        set_err(h, "a step kernel gave up waiting for its staged data (status %d)", kstatus);
        return LBM_ERR_TIMEOUT;
    }
    out[0] = fixed_to_double(r.limb) + (double)h->n_fluid * h->p.rho0;
    out[1] = r.mx;
    out[2] = r.my;
    out[3] = r.en;
    out[4] = (have && r.ures > 0.0)
                 ? std::sqrt(r.dres) / ((double)(h->steps - h->prev_step) * std::sqrt(r.ures))
                 : -1.0;
    out[5] = (double)r.nonfinite;
    out[6] = (double)h->steps;
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
    if (!h || !host) return LBM_ERR_INVALID;
    if (bytes != buf_bytes(h)) {
        set_err(h, "state buffer is %zu bytes, expected %zu", bytes, buf_bytes(h));
        return LBM_ERR_STATE;
    }
    CK(h, cudaMemcpyAsync(h->f[h->cur], host, bytes, cudaMemcpyHostToDevice, h->stream),
       "cudaMemcpyAsync(H2D)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    reset_counters(h);
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
    cudaError_t e = h->p.precision == 64
                        ? lbm::launch_diag<double>((const double*)h->f[h->cur], a, uref, have,
                                                   part, h->diag_blocks, h->stream)
                        : lbm::launch_diag<float>((const float*)h->f[h->cur], a, uref, have,
                                                  part, h->diag_blocks, h->stream);
    CK(h, e, "diagnostics kernels");
    DiagPartial r;
    CK(h, cudaMemcpyAsync(&r, part + h->diag_blocks, sizeof(r), cudaMemcpyDeviceToHost,
                          h->stream),
       "cudaMemcpyAsync(D2H)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    out[0] = fixed_to_double(r.limb) + (double)h->n_fluid * h->p.rho0;
    out[1] = r.mx;
    out[2] = r.my;
    out[3] = r.en;
    out[4] = (have && r.ures > 0.0)
                 ? std::sqrt(r.dres) / ((double)(h->steps - d.step) * std::sqrt(r.ures))
                 : -1.0;
    out[5] = (double)r.nonfinite;
    out[6] = (double)h->steps;
    d.owner = h->serial;
    d.step = h->steps;
    if (r.nonfinite > 0) {
        out[0] = NAN;
        set_err(h, "%lld fluid cells hold non-finite values", (long long)r.nonfinite);
        return LBM_ERR_UNSTABLE;
    }
    return LBM_OK;
}
