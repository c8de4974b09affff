// C ABI of the library (declared in include/lbm.h): handle management,
// argument checking, state bookkeeping (A/B current grid, AA parity, step
// counter) and dispatch to the kernels.  Host code only.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbm.h"
#include "lbm_device.cuh"
#include "lbm_launch.h"

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0;
    int stencil = LBM_D3Q19;
    int equilibrium = LBM_EQ_IMPROVED, collision = LBM_SRT, precision = LBM_F32;
    double tau = 1.0, magic = 3.0 / 16.0;
    double omega_bulk = 1.0, omega_4 = 1.0;  // MRT only
    double accel[3] = {0.0, 0.0, 0.0};
    int walls[3] = {0, 0, 0};
    int rho0_mode = 0;
    int pattern = LBM_PATTERN_AB;
    int bx = 128, by = 2;
    int cells_x = 1;
    int graphs = 1;                                // replay GRAPH_STEPS-step CUDA graphs in lbm_step
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // by starting A/B grid or AA parity
    void *a = nullptr, *b = nullptr;
    double *scratch = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false, initialised = false;
    int cur = 0;     // A/B: 0 -> a holds the current state, 1 -> b
    int parity = 0;  // AA: number of AA steps since init, mod 2
    long long t = 0;
    // adjoint sums (LBM_OPT_ADJ_DEFER_SUM): the step whose block partials wait in
    // scratch buffer adj_buf to be added to adj_pending_grad
    int adj_defer = 0;
    bool adj_pending = false;
    int adj_buf = 0;
    double *adj_pending_grad = nullptr;
    std::string err;
};

namespace {

int fail(lbm_handle h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(lbm_handle h, cudaError_t e, const char *where)
{
    return fail(h, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t elem_size(int precision)
{
    switch (precision) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    case LBM_F16S:
    case LBM_BF16S: return 2;
    }
    return 0;
}

long long ncell(const lbm_ctx *h) { return (long long)h->nx * h->ny * h->nz; }

lbm::Geo geo(const lbm_ctx *h)
{
    lbm::Geo g;
    g.nx = h->nx;
    g.ny = h->ny;
    g.nz = h->nz;
    g.wall_x = h->walls[0];
    g.wall_y = h->walls[1];
    g.wall_z = h->walls[2];
    g.ncell = ncell(h);
    return g;
}

double omega_minus(const lbm_ctx *h)
{
    if (h->collision == LBM_SRT) return 1.0 / h->tau;
    return 1.0 / (0.5 + h->magic / (h->tau - 0.5));
}

lbm::CollBoth coll(const lbm_ctx *h)
{
    lbm::CollBoth c;
    c.omega_p = 1.0 / h->tau;
    c.omega_m = omega_minus(h);
    c.kappa = h->equilibrium == LBM_EQ_IMPROVED ? 1.0 : 0.0;
    c.mrt = h->collision == LBM_MRT;
    c.omega_bulk = c.mrt ? h->omega_bulk : c.omega_p;
    c.omega_4 = c.mrt ? h->omega_4 : c.omega_p;
    for (int i = 0; i < 3; ++i) c.half_a[i] = 0.5 * h->accel[i];
    // (1 - omega-/2) F_q with F_q = w_q c_q . a / c_s^2 (Buick-Greated), for
    // the first member q = 2k+1 of each opposite pair.
    for (int k = 0; k < 9; ++k) {
        const int q = 2 * k + 1;
        const double w = lbm::WQ<double>(q);
        const double ca = lbm::CX(q) * h->accel[0] + lbm::CY(q) * h->accel[1] + lbm::CZ(q) * h->accel[2];
        c.force[k] = (1.0 - 0.5 * c.omega_m) * 3.0 * w * ca;
    }
    c.rho0_is_rho = h->rho0_mode;
    return c;
}

int layout(const lbm_ctx *h)
{
    if (h->pattern == LBM_PATTERN_AB) return lbm::AB;
    return h->parity ? lbm::AA_ODD : lbm::AA_EVEN;
}

void *current(const lbm_ctx *h) { return (h->pattern == LBM_PATTERN_AB && h->cur) ? h->b : h->a; }

bool aligned(const void *p) { return ((uintptr_t)p & 255u) == 0; }

size_t scratch_doubles(const lbm_ctx *h)
{
    lbm::Geo g = geo(h);
    size_t red = (size_t)lbm::reduce_blocks() * 8 + 8;
    size_t adj = (size_t)lbm::adjoint_blocks(g) * 2 * 2;  // two buffers of block partials (deferred sums)
    return red > adj ? red : adj;
}

// Block-partial buffer i of the adjoint step in scratch.
double *adj_partials(const lbm_ctx *h, int i) { return h->scratch + (size_t)i * 2 * lbm::adjoint_blocks(geo(h)); }

// Adds a deferred adjoint step's partials to its grad_omega (LBM_OPT_ADJ_DEFER_SUM).
int adj_flush(lbm_ctx *h, const char *where)
{
    if (!h->adj_pending) return LBM_OK;
    h->adj_pending = false;
    cudaError_t e = lbm::launch_adjoint_flush(h->precision, adj_partials(h, h->adj_buf), h->adj_pending_grad, geo(h),
                                              h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, where);
    return LBM_OK;
}

int check_ready(lbm_handle h)
{
    if (!h) return LBM_EINVAL;
    if (!h->bound) return fail(h, LBM_ESTATE, "no device memory bound (call lbm_bind first)");
    return LBM_OK;
}

int d3q19_only(lbm_handle h, const char *what)
{
    if (h->stencil == LBM_D3Q19) return LBM_OK;
    return fail(h, LBM_EUNSUPPORTED, std::string(what) + " is implemented for D3Q19 only");
}

int no_mrt(lbm_handle h, const char *what)
{
    if (h->collision != LBM_MRT) return LBM_OK;
    return fail(h, LBM_EUNSUPPORTED, std::string(what) + " supports SRT and TRT only");
}

// Address through which the kernels reach a macroscopic field buffer: device
// (or managed) memory as it is; pinned host memory through its mapped device
// address, so that lbm_init and lbm_moments read and write host buffers
// directly over the host link (no staging copy, no device allocation);
// pageable host memory is refused.  NULL stays NULL.
int field_address(lbm_handle h, const void *p, const char *name, const void **out)
{
    *out = nullptr;
    if (!p) return LBM_OK;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) return cuda_fail(h, e, name);
    switch (a.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
        *out = p;
        return LBM_OK;
    case cudaMemoryTypeHost:
        if (!a.devicePointer)
            return fail(h, LBM_EINVAL, std::string(name) + ": pinned host memory without a device mapping");
        *out = a.devicePointer;
        return LBM_OK;
    default:
        return fail(h, LBM_EINVAL, std::string(name) + ": pageable host memory (pass device memory or pinned "
                                                       "host memory)");
    }
}

int check_dtype(lbm_handle h, int dtype)
{
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(h, LBM_EINVAL, "dtype must be LBM_DTYPE_F64 or LBM_DTYPE_F32");
    return LBM_OK;
}

// One time step on stream st from the A/B grid `cur` or AA parity `parity`,
// which are advanced on success.
cudaError_t launch_one(const lbm_ctx *h, cudaStream_t st, int &cur, int &parity, const lbm::Geo &g,
                       const lbm::CollBoth &c, const lbm::LaunchShape &shape)
{
    cudaError_t e;
    if (h->pattern == LBM_PATTERN_AB) {
        void *src = cur ? h->b : h->a;
        void *dst = cur ? h->a : h->b;
        e = h->stencil == LBM_D3Q27 ? lbm::launch_step27(h->precision, src, dst, g, c, shape, st)
                                    : lbm::launch_step(h->precision, 0, src, dst, g, c, shape, st);
        if (e == cudaSuccess) cur ^= 1;
    } else {
        e = lbm::launch_step(h->precision, parity ? 2 : 1, h->a, h->a, g, c, shape, st);
        if (e == cudaSuccess) parity ^= 1;
    }
    return e;
}

// Steps per CUDA graph: even, so that a replay returns to the grid (A/B) or
// parity (AA) it started from.
constexpr int GRAPH_STEPS = 16;

void drop_graphs(lbm_ctx *h)
{
    for (int i = 0; i < 2; ++i) {
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
        h->gexec[i] = nullptr;
    }
}

// Captures GRAPH_STEPS steps starting from `slot` (A/B grid or AA parity) on
// a private stream (thread-local capture mode, so other threads' work is not
// affected) and instantiates them.
cudaError_t build_graph(lbm_ctx *h, int slot, const lbm::Geo &g, const lbm::CollBoth &c,
                        const lbm::LaunchShape &shape)
{
    cudaStream_t ps = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int cur = slot, parity = slot;
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < GRAPH_STEPS && le == cudaSuccess; ++k) le = launch_one(h, ps, cur, parity, g, c, shape);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(ps, &graph);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[slot], graph, 0);
        if (graph) cudaGraphDestroy(graph);
    }
    cudaStreamDestroy(ps);
    if (e != cudaSuccess) h->gexec[slot] = nullptr;
    return e;
}

}  // namespace

extern "C" {

int lbm_abi_version(void) { return LBM_ABI_VERSION; }

const char *lbm_status_string(int s)
{
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of host memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSUPPORTED: return "unsupported";
    case LBM_ENONFINITE: return "non-finite populations";
    case LBM_ESTATE: return "call out of order";
    }
    return "unknown status";
}

int lbm_velocity_set(int *c, double *w, int *opp)
{
    for (int q = 0; q < lbm::Q; ++q) {
        if (c) {
            c[3 * q + 0] = lbm::CX(q);
            c[3 * q + 1] = lbm::CY(q);
            c[3 * q + 2] = lbm::CZ(q);
        }
        if (w) w[q] = lbm::WQ<double>(q);
        if (opp) opp[q] = lbm::OPP(q);
    }
    return LBM_OK;
}

int lbm_velocity_set_of(int stencil, int *c, double *w, int *opp)
{
    if (stencil == LBM_D3Q19) return lbm_velocity_set(c, w, opp);
    if (stencil == LBM_D3Q27) {
        lbm::velocity_set27(c, w, opp);
        return LBM_OK;
    }
    return LBM_EUNSUPPORTED;
}

int lbm_create(int nx, int ny, int nz, int stencil, int equilibrium, int collision, double tau, int precision,
               lbm_handle *out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nz > 65535) return LBM_EINVAL;
    if ((long long)nx * ny * nz >= (1LL << 31)) return LBM_EUNSUPPORTED;
    if (stencil != LBM_D3Q19 && stencil != LBM_D3Q27) return LBM_EUNSUPPORTED;
    if (equilibrium != LBM_EQ_STANDARD && equilibrium != LBM_EQ_IMPROVED) return LBM_EINVAL;
    if (collision != LBM_SRT && collision != LBM_TRT && collision != LBM_MRT) return LBM_EINVAL;
    if (collision == LBM_MRT && stencil != LBM_D3Q19) return LBM_EUNSUPPORTED;
    if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;
    if (elem_size(precision) == 0) return LBM_EINVAL;
    lbm_ctx *h = new (std::nothrow) lbm_ctx();
    if (!h) return LBM_ENOMEM;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->stencil = stencil;
    h->equilibrium = equilibrium;
    h->collision = collision;
    h->tau = tau;
    h->precision = precision;
    if (nx < 128) {
        h->bx = nx <= 32 ? 32 : (nx <= 64 ? 64 : 128);
        h->by = 256 / h->bx;
    }
    // 16-bit storage needs wide accesses shared by several cells to approach
    // the bandwidth roofline: four cells per thread (A/B and AA)
    h->cells_x = (precision == LBM_F16S || precision == LBM_BF16S) ? 4 : 1;
    *out = h;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    if (!h) return LBM_EINVAL;
    drop_graphs(h);
    delete h;
    return LBM_OK;
}

int lbm_set_option(lbm_handle h, int key, double v)
{
    if (!h) return LBM_EINVAL;
    if (!std::isfinite(v)) return fail(h, LBM_EINVAL, "option value must be finite");
    drop_graphs(h);  // captured kernels carry the old parameters
    switch (key) {
    case LBM_OPT_TRT_MAGIC:
        if (!(v > 0)) return fail(h, LBM_EINVAL, "TRT magic parameter must be > 0");
        h->magic = v;
        return LBM_OK;
    case LBM_OPT_FORCE_X:
    case LBM_OPT_FORCE_Y:
    case LBM_OPT_FORCE_Z: h->accel[key - LBM_OPT_FORCE_X] = v; return LBM_OK;
    case LBM_OPT_WALLS_X:
    case LBM_OPT_WALLS_Y:
    case LBM_OPT_WALLS_Z:
        if (v != 0.0 && v != 1.0) return fail(h, LBM_EINVAL, "walls option must be 0 or 1");
        h->walls[key - LBM_OPT_WALLS_X] = (int)v;
        return LBM_OK;
    case LBM_OPT_RHO0_MODE:
        if (v != 0.0 && v != 1.0) return fail(h, LBM_EINVAL, "rho0 mode must be 0 or 1");
        h->rho0_mode = (int)v;
        return LBM_OK;
    case LBM_OPT_PATTERN:
        if (v != LBM_PATTERN_AB && v != LBM_PATTERN_AA) return fail(h, LBM_EINVAL, "pattern must be AB or AA");
        if (v == LBM_PATTERN_AA && h->stencil == LBM_D3Q27)
            return fail(h, LBM_EUNSUPPORTED, "the AA pattern is D3Q19 only");
        if ((int)v != h->pattern) {
            h->pattern = (int)v;
            h->initialised = false;
            h->cur = 0;
            h->parity = 0;
        }
        return LBM_OK;
    case LBM_OPT_TAU:
        if (!(v > 0.5)) return fail(h, LBM_EINVAL, "tau must be > 1/2");
        h->tau = v;
        return LBM_OK;
    case LBM_OPT_EQUILIBRIUM:
        if (v != LBM_EQ_STANDARD && v != LBM_EQ_IMPROVED) return fail(h, LBM_EINVAL, "bad equilibrium");
        h->equilibrium = (int)v;
        return LBM_OK;
    case LBM_OPT_COLLISION:
        if (v != LBM_SRT && v != LBM_TRT && v != LBM_MRT) return fail(h, LBM_EINVAL, "bad collision");
        if (v == LBM_MRT && h->stencil != LBM_D3Q19) return fail(h, LBM_EUNSUPPORTED, "MRT is D3Q19 only");
        h->collision = (int)v;
        return LBM_OK;
    case LBM_OPT_MRT_OMEGA_BULK:
    case LBM_OPT_MRT_OMEGA_4:
        if (!(v > 0.0 && v < 2.0)) return fail(h, LBM_EINVAL, "MRT rates must lie in (0, 2)");
        (key == LBM_OPT_MRT_OMEGA_BULK ? h->omega_bulk : h->omega_4) = v;
        return LBM_OK;
    case LBM_OPT_GRAPHS:
        if (v != 0.0 && v != 1.0) return fail(h, LBM_EINVAL, "graphs option must be 0 or 1");
        h->graphs = (int)v;
        return LBM_OK;
    case LBM_OPT_ADJ_DEFER_SUM: {
        if (v != 0.0 && v != 1.0) return fail(h, LBM_EINVAL, "deferred adjoint sums option must be 0 or 1");
        const int st = adj_flush(h, "lbm_set_option (adjoint flush)");
        h->adj_defer = (int)v;
        return st;
    }
    case LBM_OPT_CELLS_X:
        if (v != 1.0 && v != 2.0 && v != 4.0) return fail(h, LBM_EINVAL, "cells per thread must be 1, 2 or 4");
        h->cells_x = (int)v;
        return LBM_OK;
    case LBM_OPT_BLOCK_X:
    case LBM_OPT_BLOCK_Y: {
        int bx = key == LBM_OPT_BLOCK_X ? (int)v : h->bx;
        int by = key == LBM_OPT_BLOCK_Y ? (int)v : h->by;
        if ((double)(int)v != v || bx < 1 || by < 1 || bx * by > 256 || (bx * by) % 32)
            return fail(h, LBM_EINVAL, "block must satisfy bx * by <= 256 and a multiple of 32");
        h->bx = bx;
        h->by = by;
        return LBM_OK;
    }
    }
    return fail(h, LBM_EINVAL, "unknown option key");
}

int lbm_get_option(lbm_handle h, int key, double *v)
{
    if (!h || !v) return LBM_EINVAL;
    switch (key) {
    case LBM_OPT_TRT_MAGIC: *v = h->magic; return LBM_OK;
    case LBM_OPT_FORCE_X:
    case LBM_OPT_FORCE_Y:
    case LBM_OPT_FORCE_Z: *v = h->accel[key - LBM_OPT_FORCE_X]; return LBM_OK;
    case LBM_OPT_WALLS_X:
    case LBM_OPT_WALLS_Y:
    case LBM_OPT_WALLS_Z: *v = h->walls[key - LBM_OPT_WALLS_X]; return LBM_OK;
    case LBM_OPT_RHO0_MODE: *v = h->rho0_mode; return LBM_OK;
    case LBM_OPT_PATTERN: *v = h->pattern; return LBM_OK;
    case LBM_OPT_TAU: *v = h->tau; return LBM_OK;
    case LBM_OPT_EQUILIBRIUM: *v = h->equilibrium; return LBM_OK;
    case LBM_OPT_COLLISION: *v = h->collision; return LBM_OK;
    case LBM_OPT_MRT_OMEGA_BULK: *v = h->omega_bulk; return LBM_OK;
    case LBM_OPT_MRT_OMEGA_4: *v = h->omega_4; return LBM_OK;
    case LBM_OPT_CELLS_X: *v = h->cells_x; return LBM_OK;
    case LBM_OPT_GRAPHS: *v = h->graphs; return LBM_OK;
    case LBM_OPT_ADJ_DEFER_SUM: *v = h->adj_defer; return LBM_OK;
    case LBM_OPT_BLOCK_X: *v = h->bx; return LBM_OK;
    case LBM_OPT_BLOCK_Y: *v = h->by; return LBM_OK;
    }
    return fail(h, LBM_EINVAL, "unknown option key");
}

int lbm_required_bytes(lbm_handle h, size_t *pdf_bytes, int *n_grids, size_t *scratch_bytes)
{
    if (!h) return LBM_EINVAL;
    if (pdf_bytes) *pdf_bytes = (size_t)h->stencil * (size_t)ncell(h) * elem_size(h->precision);
    if (n_grids) *n_grids = h->pattern == LBM_PATTERN_AB ? 2 : 1;
    if (scratch_bytes) *scratch_bytes = ((scratch_doubles(h) * sizeof(double) + 255) / 256) * 256;
    return LBM_OK;
}

int lbm_bind(lbm_handle h, void *pdf_a, void *pdf_b, void *scratch, void *stream)
{
    if (!h) return LBM_EINVAL;
    if (!pdf_a) return fail(h, LBM_EINVAL, "pdf_a is NULL");
    if (h->pattern == LBM_PATTERN_AB && !pdf_b) return fail(h, LBM_EINVAL, "A/B pattern needs pdf_b");
    if (h->pattern == LBM_PATTERN_AB && pdf_a == pdf_b) return fail(h, LBM_EINVAL, "pdf_a and pdf_b must differ");
    if (!aligned(pdf_a) || (pdf_b && !aligned(pdf_b)) || (scratch && !aligned(scratch)))
        return fail(h, LBM_EINVAL, "device buffers must be 256-byte aligned");
    if ((double *)scratch != h->scratch || (cudaStream_t)stream != h->stream) {
        const int st = adj_flush(h, "lbm_bind (adjoint flush)");  // pending partials live in the old scratch
        if (st) return st;
    }
    drop_graphs(h);  // captured kernels carry the old grid pointers
    h->a = pdf_a;
    h->b = h->pattern == LBM_PATTERN_AB ? pdf_b : nullptr;
    h->scratch = (double *)scratch;
    h->stream = (cudaStream_t)stream;
    h->cur = 0;
    h->bound = true;
    return LBM_OK;
}

int lbm_init(lbm_handle h, const void *rho, const void *u, int dtype)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = check_dtype(h, dtype))) return s;
    if (!u) return fail(h, LBM_EINVAL, "u is NULL");
    const void *rho_d, *u_d;
    if ((s = field_address(h, rho, "lbm_init rho", &rho_d))) return s;
    if ((s = field_address(h, u, "lbm_init u", &u_d))) return s;
    rho = rho_d;
    u = u_d;
    h->parity = 0;
    cudaError_t e = h->stencil == LBM_D3Q27
                        ? lbm::launch_init27(h->precision, current(h), rho, u, dtype, geo(h), coll(h), h->stream)
                        : lbm::launch_init(h->precision, layout(h), current(h), rho, u, dtype, geo(h), coll(h),
                                           h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_init");
    h->t = 0;
    h->initialised = true;
    return LBM_OK;
}

int lbm_step(lbm_handle h, int n)
{
    int s = check_ready(h);
    if (s) return s;
    if (n < 0) return fail(h, LBM_EINVAL, "n must be >= 0");
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised (lbm_init or lbm_set_pdfs)");
    const lbm::Geo g = geo(h);
    const lbm::CollBoth c = coll(h);
    const lbm::LaunchShape shape{h->bx, h->by, h->cells_x};
    int i = 0;
    if (h->graphs && n >= GRAPH_STEPS) {
        // Replay whole graphs of GRAPH_STEPS steps (one launch call for many
        // kernels), unless the caller is capturing the bound stream itself:
        // then the plain launches below are recorded into the caller's graph.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(h->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            const int slot = h->pattern == LBM_PATTERN_AB ? h->cur : h->parity;
            if (!h->gexec[slot] && build_graph(h, slot, g, c, shape) != cudaSuccess) {
                cudaGetLastError();  // capture failed: step without graphs
                h->graphs = 0;
            }
            if (h->gexec[slot]) {
                for (; i + GRAPH_STEPS <= n; i += GRAPH_STEPS) {
                    cudaError_t e = cudaGraphLaunch(h->gexec[slot], h->stream);
                    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step (graph)");
                    h->t += GRAPH_STEPS;
                }
            }
        }
    }
    for (; i < n; ++i) {
        cudaError_t e = launch_one(h, h->stream, h->cur, h->parity, g, c, shape);
        if (e != cudaSuccess) return cuda_fail(h, e, "lbm_step");
        ++h->t;
    }
    return LBM_OK;
}

int lbm_moments(lbm_handle h, void *rho, void *u, int dtype)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = check_dtype(h, dtype))) return s;
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised");
    if (!rho && !u) return LBM_OK;
    const void *rho_d, *u_d;
    if ((s = field_address(h, rho, "lbm_moments rho", &rho_d))) return s;
    if ((s = field_address(h, u, "lbm_moments u", &u_d))) return s;
    rho = const_cast<void *>(rho_d);
    u = const_cast<void *>(u_d);
    cudaError_t e = h->stencil == LBM_D3Q27
                        ? lbm::launch_moments27(h->precision, current(h), rho, u, dtype, geo(h), coll(h), h->stream)
                        : lbm::launch_moments(h->precision, layout(h), current(h), rho, u, dtype, geo(h), coll(h),
                                              h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_moments");
    return LBM_OK;
}

int lbm_reduce(lbm_handle h, double *out)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_reduce"))) return s;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!h->scratch) return fail(h, LBM_ESTATE, "lbm_reduce needs a scratch buffer (lbm_bind)");
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised");
    if ((s = adj_flush(h, "lbm_reduce (adjoint flush)"))) return s;  // the reduction reuses the scratch
    double *result = h->scratch + (size_t)lbm::reduce_blocks() * 8;
    cudaError_t e = lbm::launch_reduce(h->precision, layout(h), current(h), h->scratch, result, geo(h), coll(h),
                                       h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce");
    e = cudaMemcpyAsync(out, result, LBM_RED_COUNT * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce copy");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce sync");
    if (out[LBM_RED_NONFINITE] > 0) return fail(h, LBM_ENONFINITE, "state holds non-finite populations");
    return LBM_OK;
}

int lbm_enstrophy(lbm_handle h, double *out)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_enstrophy"))) return s;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!h->scratch) return fail(h, LBM_ESTATE, "lbm_enstrophy needs a scratch buffer (lbm_bind)");
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised");
    if ((s = adj_flush(h, "lbm_enstrophy (adjoint flush)"))) return s;  // the reduction reuses the scratch
    double *result = h->scratch + (size_t)lbm::reduce_blocks() * 8;
    cudaError_t e = lbm::launch_enstrophy(h->precision, layout(h), current(h), h->scratch, result, geo(h), coll(h),
                                          h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_enstrophy");
    e = cudaMemcpyAsync(out, result, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_enstrophy copy");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_enstrophy sync");
    if (!std::isfinite(*out)) return fail(h, LBM_ENONFINITE, "enstrophy is not finite");
    return LBM_OK;
}

int lbm_reduce_noalloc(lbm_handle h, double *out)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_reduce_noalloc"))) return s;
    if (!out) return fail(h, LBM_EINVAL, "out is NULL");
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised");
    if ((long long)lbm::reduce_blocks() * 8 + 8 > lbm::reduce_noalloc_capacity_doubles())
        return fail(h, LBM_EUNSUPPORTED, "lbm_reduce_noalloc: the reduction needs more partial rows than the "
                                         "static scratch array holds");
    double *result = nullptr;
    cudaError_t e = lbm::launch_reduce_noalloc(h->precision, layout(h), current(h), geo(h), coll(h), h->stream,
                                               &result);
    if (e == cudaErrorInvalidDevice)
        return fail(h, LBM_EINVAL, "lbm_reduce_noalloc: the calling thread's current device is not the device of "
                                   "the bound stream");
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce_noalloc");
    e = cudaMemcpyAsync(out, result, LBM_RED_COUNT * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce_noalloc copy");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_reduce_noalloc sync");
    if (out[LBM_RED_NONFINITE] > 0) return fail(h, LBM_ENONFINITE, "state holds non-finite populations");
    return LBM_OK;
}

int lbm_steps_done(lbm_handle h, long long *t)
{
    if (!h || !t) return LBM_EINVAL;
    *t = h->t;
    return LBM_OK;
}

int lbm_get_pdfs(lbm_handle h, void *dst)
{
    int s = check_ready(h);
    if (s) return s;
    if (!dst) return fail(h, LBM_EINVAL, "dst is NULL");
    if (!h->initialised) return fail(h, LBM_ESTATE, "state not initialised");
    if (dst == h->a || (h->b && dst == h->b)) return fail(h, LBM_EINVAL, "dst must not be a bound grid");
    cudaError_t e = h->stencil == LBM_D3Q27
                        ? lbm::launch_get27(h->precision, current(h), dst, geo(h), h->stream)
                        : lbm::launch_get_pdfs(h->precision, layout(h), current(h), dst, geo(h), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_get_pdfs");
    return LBM_OK;
}

int lbm_set_pdfs(lbm_handle h, const void *src)
{
    int s = check_ready(h);
    if (s) return s;
    if (!src) return fail(h, LBM_EINVAL, "src is NULL");
    if (src == h->a || (h->b && src == h->b)) return fail(h, LBM_EINVAL, "src must not be a bound grid");
    h->parity = 0;
    cudaError_t e = h->stencil == LBM_D3Q27
                        ? lbm::launch_set27(h->precision, current(h), src, geo(h), h->stream)
                        : lbm::launch_set_pdfs(h->precision, layout(h), current(h), src, geo(h), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_set_pdfs");
    h->t = 0;
    h->initialised = true;
    return LBM_OK;
}

int lbm_adjoint_seed(lbm_handle h, const void *grad_rho, const void *grad_u, int dtype, void *lambda)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_adjoint_seed"))) return s;
    if ((s = no_mrt(h, "lbm_adjoint_seed"))) return s;
    if ((s = check_dtype(h, dtype))) return s;
    if (h->rho0_mode) return fail(h, LBM_EUNSUPPORTED, "adjoint supports rho0 = 1 only");
    if (!grad_u || !lambda) return fail(h, LBM_EINVAL, "grad_u and lambda are required");
    if ((s = adj_flush(h, "lbm_adjoint_seed (adjoint flush)"))) return s;
    cudaError_t e = lbm::launch_adjoint_seed(h->precision, grad_rho, grad_u, dtype, lambda, geo(h), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_adjoint_seed");
    return LBM_OK;
}

int lbm_adjoint_step(lbm_handle h, const void *state_t, const void *lambda_next, void *lambda_t, double *grad_omega)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_adjoint_step"))) return s;
    if ((s = no_mrt(h, "lbm_adjoint_step"))) return s;
    if (h->rho0_mode) return fail(h, LBM_EUNSUPPORTED, "adjoint supports rho0 = 1 only");
    if (!state_t || !lambda_next || !lambda_t || !grad_omega) return fail(h, LBM_EINVAL, "null argument");
    if (lambda_next == lambda_t) return fail(h, LBM_EINVAL, "lambda_next and lambda_t must differ");
    if (!h->scratch) return fail(h, LBM_ESTATE, "lbm_adjoint_step needs a scratch buffer (lbm_bind)");
    cudaError_t e;
    if (!h->adj_defer) {
        e = lbm::launch_adjoint_step(h->precision, state_t, lambda_next, lambda_t, grad_omega, adj_partials(h, 0),
                                     nullptr, nullptr, false, geo(h), coll(h), h->stream);
    } else {
        // this step's partials go to the other buffer; the pending step's are summed by this step's first block
        const int buf = h->adj_pending ? 1 - h->adj_buf : 0;
        e = lbm::launch_adjoint_step(h->precision, state_t, lambda_next, lambda_t, grad_omega, adj_partials(h, buf),
                                     h->adj_pending ? adj_partials(h, h->adj_buf) : nullptr,
                                     h->adj_pending ? h->adj_pending_grad : nullptr, true, geo(h), coll(h),
                                     h->stream);
        h->adj_pending = e == cudaSuccess;
        h->adj_buf = buf;
        h->adj_pending_grad = grad_omega;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_adjoint_step");
    return LBM_OK;
}

int lbm_adjoint_flush(lbm_handle h)
{
    int s = check_ready(h);
    if (s) return s;
    return adj_flush(h, "lbm_adjoint_flush");
}

int lbm_adjoint_init_velocity(lbm_handle h, const void *rho, const void *u0, int dtype, const void *lambda0,
                              void *grad_u0)
{
    int s = check_ready(h);
    if (s) return s;
    if ((s = d3q19_only(h, "lbm_adjoint_init_velocity"))) return s;
    if ((s = no_mrt(h, "lbm_adjoint_init_velocity"))) return s;
    if ((s = check_dtype(h, dtype))) return s;
    if (h->rho0_mode) return fail(h, LBM_EUNSUPPORTED, "adjoint supports rho0 = 1 only");
    if (!u0 || !lambda0 || !grad_u0) return fail(h, LBM_EINVAL, "null argument");
    cudaError_t e = lbm::launch_adjoint_init_velocity(h->precision, rho, u0, dtype, lambda0, grad_u0, geo(h), coll(h),
                                                      h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbm_adjoint_init_velocity");
    return LBM_OK;
}

int lbm_adjoint_tau_gradient(lbm_handle h, const double *grad_omega, double *dL_dtau)
{
    if (!h || !grad_omega || !dL_dtau) return LBM_EINVAL;
    int s = no_mrt(h, "lbm_adjoint_tau_gradient");
    if (s) return s;
    const double tau = h->tau;
    const double dwp = -1.0 / (tau * tau);
    double dwm = dwp;
    if (h->collision == LBM_TRT) {
        const double tm = 0.5 + h->magic / (tau - 0.5);
        const double dtm = -h->magic / ((tau - 0.5) * (tau - 0.5));
        dwm = -dtm / (tm * tm);
    }
    *dL_dtau = grad_omega[0] * dwp + grad_omega[1] * dwm;
    return LBM_OK;
}

const char *lbm_last_error(lbm_handle h)
{
    if (!h) return "invalid handle";
    return h->err.c_str();
}

}  // extern "C"
